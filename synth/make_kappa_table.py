"""Write synth/kappa_table.json: kappa with min|eig(gamma5 D)| = 1e-3 per lattice.

Calls only the FP64 oracle (oracle.kappa): a dense eigensolve for lattices
of at most 256 sites, thick-restart Lanczos on D^dagger D otherwise.

    python synth/make_kappa_table.py 4x4x4x4:1 16x16x16x32:2
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import synth  # noqa: E402
from oracle import kappa as okappa  # noqa: E402


def main(argv):
    table = {}
    if os.path.exists(synth.KAPPA_TABLE):
        with open(synth.KAPPA_TABLE) as f:
            table = json.load(f)
    for spec in argv:
        lat, seed = spec.split(":")
        dims = tuple(int(v) for v in lat.split("x"))
        seed = int(seed)
        U = synth.su3_links(dims, seed)
        t0 = time.time()
        if synth.volume(dims) <= 256:
            kap, sig = okappa.kappa_dense(U, dims)
            how = "dense LAPACK eigvalsh of D^dagger D; scan from 0 by 0.005, Illinois refine"
        else:
            start = float(os.environ.get("KAPPA_START", "0.262"))
            step = float(os.environ.get("KAPPA_STEP", "0.003"))
            rtol = float(os.environ.get("KAPPA_RTOL", "1e-3"))
            cap = int(os.environ.get("KAPPA_MAX_CYCLES", "2000"))
            kap, sig, res = okappa.kappa_iterative(
                U, dims, start=start, step=step, rtol=rtol, max_cycles=cap,
                log=lambda s: print(s, flush=True))
            how = ("MinRes-DR(100,20) as an eigensolver: harmonic Ritz pair nearest zero of "
                   f"gamma5 D (at most {cap} cycles per evaluation); steps of {step} from {start} "
                   f"to bracket, Illinois refine to |sigma/1e-3 - 1| < {rtol}; harmonic Ritz "
                   f"residual of the final estimate {res:.2e}")
        key = f"{lat}_s{seed}"
        table[key] = dict(kappa=kap, sigma_min=sig, method=how,
                          seconds=round(time.time() - t0, 1), host=platform.machine())
        print(key, table[key], flush=True)
        with open(synth.KAPPA_TABLE, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
