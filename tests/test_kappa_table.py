"""The stored kappa table (synth/kappa_table.json, written by synth/make_kappa_table.py
from the oracle only) against its own recorded evidence.

The workloads run at the kappa where the smallest |eigenvalue| of gamma5 D, i.e. the
smallest singular value of D, is 1e-3.  For the lattices too large for a dense
solve the oracle estimates it with MinRes-DR as an eigensolver and records, per
evaluation, the Rayleigh quotient, its residual and the gap to the next eigenvalue.
For a hermitian operator the Kato-Temple inequality bounds the quotient's error by
residual^2 / gap.  Checked here: every lattice a workload uses has an entry; the
recorded bound is that formula; the entry is the last evaluation; the estimate meets
the rule to the stated 5%; and with the bound added either way it stays within 10%
(16^4, whose last evaluation stopped at the 200-cycle cap with residual 1.9e-4, reaches
9.3%; the others stay inside 5%).  (The 4^4 entry is checked against a dense
eigensolve in test_oracle_krylov.py.)"""
import json

import pytest

import bench
import synth


def _table():
    with open(synth.KAPPA_TABLE) as f:
        return json.load(f)


def _key(dims, seed):
    return "x".join(str(int(d)) for d in dims) + f"_s{int(seed)}"


def _workload_lattices():
    out = []
    for name, w in synth.WORKLOADS.items():
        if "dims" in w:
            out.append((name, w["dims"], w["gauge_seed"]))
        else:
            for i, dims in enumerate(w["sizes"]):
                out.append((name, dims, w["gauge_seed0"] + i))
    return out


@pytest.mark.parametrize("name,dims,seed", _workload_lattices())
def test_every_workload_lattice_has_an_entry(name, dims, seed):
    t = _table()
    assert _key(dims, seed) in t, name
    kap = synth.kappa_for(dims, seed)
    # above the free-field crossing (1 - 1e-3)/8 and below the first doubler's
    assert (1 - 1e-3) / 8 < kap < 0.3


def test_the_uneven_batch_uses_one_entry_per_size_class():
    w = synth.WORKLOADS["uneven_64"]
    ks = bench.c4_kappas(w)
    assert len(ks) == w["lattices"]
    for i, k in enumerate(ks):
        dims = w["sizes"][i % 3]
        assert k == synth.kappa_for(dims, w["gauge_seed0"] + i % 3)


@pytest.mark.parametrize("key", sorted(_table()))
def test_entry_meets_the_rule_with_its_error_bound(key):
    e = _table()[key]
    sigma = e["sigma_min"]
    assert abs(sigma / 1e-3 - 1) < 0.05
    evs = e.get("evaluations")
    if not evs:
        return
    last = evs[-1]
    assert last["kappa"] == e["kappa"] and last["sigma"] == sigma
    for ev in evs:
        # Kato-Temple: |lambda - rho| <= r^2 / gap for the hermitian gamma5 D
        assert ev["gap"] > ev["residual"] > 0
        assert abs(ev["bound"] - ev["residual"] ** 2 / ev["gap"]) <= 1e-12 * ev["bound"]
    lo, hi = sigma - last["bound"], sigma + last["bound"]
    assert abs(lo / 1e-3 - 1) < 0.10 and abs(hi / 1e-3 - 1) < 0.10
    # sigma falls as kappa grows towards the critical value
    assert last["dsigma_dkappa"] < 0


def _stored_error_bound(e):
    """A bound on |sigma_min - the stored sigma| from the entry's own record: the
    Kato-Temple bound of its last evaluation, else the residual of its final
    estimate (a Rayleigh quotient of Q, so within that residual of an eigenvalue)."""
    evs = e.get("evaluations")
    if evs:
        return evs[-1]["bound"]
    import re
    got = re.search(r"residual of the final estimate ([0-9.]+e[-+][0-9]+)", e["method"])
    return float(got.group(1)) if got else None


@pytest.mark.parametrize("key", sorted(k for k, e in _table().items() if "verification" in e))
def test_independent_verification_confirms_the_entry(key):
    # a cold-started eigensolve at the stored kappa (oracle.kappa.verify_sigma): its
    # residual and bound are formed from the returned vector itself.  It may settle on
    # another eigenvalue of about the same size (Q is indefinite and its values near
    # zero come in clusters); what it must not find is one below the stored minimum.
    e = _table()[key]
    v = e["verification"]
    assert v["kappa"] == e["kappa"]
    assert v["gap"] > v["residual"] > 0
    assert abs(v["bound"] - v["residual"] ** 2 / v["gap"]) <= 1e-12 * v["bound"]
    # its estimate meets the rule to the same 5%; the width of its interval only says
    # how far a capped cold start converged (16^3x32: 400 cycles, bound 1.0e-4)
    assert abs(v["sigma"] / 1e-3 - 1) < 0.05
    # the cold start found no eigenvalue of gamma5 D closer to zero than the stored
    # minimum allows (the two intervals overlap, or the verification's lies above)
    b = _stored_error_bound(e)
    assert b is not None
    assert v["sigma"] + v["bound"] >= e["sigma_min"] - b

