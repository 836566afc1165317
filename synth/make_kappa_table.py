"""Write synth/kappa_table.json: kappa with min|eig(gamma5 D)| = 1e-3 per lattice.

Calls only the FP64 oracle (oracle.kappa): a dense eigensolve for lattices
of at most 256 sites, thick-restart Lanczos on D^dagger D otherwise.

    python synth/make_kappa_table.py 4x4x4x4:1 16x16x16x32:2

With --verify the stored kappa of each named lattice is re-verified by one
independent, cold-started eigensolve at that kappa (oracle.kappa.verify_sigma);
the result is stored beside the entry as "verification" and the kappa itself is
left as it is:

    KAPPA_VERIFY_CYCLES=150 python synth/make_kappa_table.py --verify 24x24x24x48:3
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


def _store(key, entry):
    """Add one entry to the table, re-reading it first (several searches may run at once)."""
    import fcntl
    with open(synth.KAPPA_TABLE + ".lock", "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        table = {}
        if os.path.exists(synth.KAPPA_TABLE):
            with open(synth.KAPPA_TABLE) as f:
                table = json.load(f)
        table[key] = entry
        tmp = synth.KAPPA_TABLE + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, synth.KAPPA_TABLE)


def verify(argv):
    seed = int(os.environ.get("KAPPA_VERIFY_SEED", "777"))
    cap = int(os.environ.get("KAPPA_VERIFY_CYCLES", "400"))
    rel = float(os.environ.get("KAPPA_VERIFY_REL", "1e-3"))
    for spec in argv:
        lat, gseed = spec.split(":")
        dims = tuple(int(v) for v in lat.split("x"))
        key = f"{lat}_s{int(gseed)}"
        with open(synth.KAPPA_TABLE) as f:
            entry = json.load(f)[key]
        U = synth.su3_links(dims, int(gseed))
        t0 = time.time()
        v = okappa.verify_sigma(U, entry["kappa"], dims, seed, rel_bound=rel, max_cycles=cap,
                                log=lambda s: print(s, flush=True))
        v["method"] = (f"MinRes-DR(100,20) as an eigensolver, cold start from a complex Gaussian "
                       f"vector (seed {seed}), at most {cap} cycles, stop at r^2/3e-4 <= {rel} |theta|; "
                       f"Rayleigh quotient and residual of the unit Ritz vector formed anew")
        v["seconds"] = round(time.time() - t0, 1)
        v["host"] = platform.machine()
        print(key, v, flush=True)
        with open(synth.KAPPA_TABLE) as f:
            entry = json.load(f)[key]
        entry["verification"] = v
        _store(key, entry)


def main(argv):
    if argv and argv[0] == "--verify":
        verify(argv[1:])
        return
    for spec in argv:
        lat, seed = spec.split(":")
        dims = tuple(int(v) for v in lat.split("x"))
        seed = int(seed)
        U = synth.su3_links(dims, seed)
        t0 = time.time()
        bracket = os.environ.get("KAPPA_BRACKET")
        if bracket:
            # a:sigma_a:b:sigma_b from earlier oracle evaluations on this lattice
            a, sa, b, sb = (float(v) for v in bracket.split(":"))
            rtol = float(os.environ.get("KAPPA_RTOL", "1e-4"))
            cap = int(os.environ.get("KAPPA_MAX_CYCLES", "150"))
            kap, sig, res, bound, hist = okappa.kappa_newton(
                U, dims, a, sa, b, sb, rtol=rtol, max_cycles=cap,
                log=lambda s: print(s, flush=True))
            how = ("MinRes-DR(100,20) as an eigensolver (Rayleigh quotient of the harmonic Ritz "
                   f"vector nearest zero, warm-started, at most {cap} cycles per evaluation); "
                   f"Newton with the Hellmann-Feynman slope inside the bracket [{a}, {b}] to "
                   f"|sigma/1e-3 - 1| < {rtol}; residual of the final estimate {res:.2e}, "
                   f"Kato-Temple bound on its error {bound:.2e}")
            extra = dict(evaluations=hist)
        elif synth.volume(dims) <= 256:
            extra = {}
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
            extra = {}
            how = ("MinRes-DR(100,20) as an eigensolver: harmonic Ritz pair nearest zero of "
                   f"gamma5 D (at most {cap} cycles per evaluation); steps of {step} from {start} "
                   f"to bracket, Illinois refine to |sigma/1e-3 - 1| < {rtol}; harmonic Ritz "
                   f"residual of the final estimate {res:.2e}")
        key = f"{lat}_s{seed}"
        entry = dict(kappa=kap, sigma_min=sig, method=how,
                     seconds=round(time.time() - t0, 1), host=platform.machine(), **extra)
        print(key, entry, flush=True)
        _store(key, entry)


if __name__ == "__main__":
    main(sys.argv[1:])
