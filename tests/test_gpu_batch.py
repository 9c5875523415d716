"""GPU parity of the batched path (many independent meshes of uneven size,
order and material in one set of launches) against the oracle, problem by
problem.  Tolerances as for a single context: float64 1e-10 for operators;
Newmark steps 1e-9 (u) / 1e-8 (v) / 1e-7 (a) at Newton 1e-12; mixed
operators 2e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import solvers  # noqa: E402
from oracle.assembly import Discretization  # noqa: E402
from oracle.basis1d import Basis1D  # noqa: E402
from oracle.hexmesh import BoxMesh  # noqa: E402
from oracle.material import lame  # noqa: E402
from synthetic import random_uniform, random_vector  # noqa: E402

TOL64, TOL32 = 1e-10, 2e-5


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _problems(seed=0, n=7, orders=(1, 2, 3, 4, 5, 8), max_e=3):
    """Seeded uneven problems: sides in 1..max_e elements, order from
    `orders`, E in [5e2, 5e3], nu in [0.25, 0.45]; bottom face clamped."""
    r = random_uniform(5 * n, seed, 0.0, 1.0).reshape(n, 5)
    out = []
    for i in range(n):
        elems = tuple(1 + int(r[i, k] * max_e) % max_e for k in range(3))
        P = orders[i % len(orders)]
        mu, lam = lame(5e2 + 4.5e3 * r[i, 3], 0.25 + 0.2 * r[i, 4])
        out.append(dict(elems=elems, lengths=(1.0, 0.8, 1.2), clamp={"zmin": (0, 1, 2)}, mu=mu, lam=lam, rho=1.0,
                        P=P))
    return out


def _oracles(probs, kind):
    ds = []
    for pr in probs:
        mesh = BoxMesh(*pr["elems"], pr["P"], lengths=pr["lengths"])
        for f, c in pr["clamp"].items():
            mesh.clamp(f, c)
        ds.append(Discretization(mesh, Basis1D(pr["P"], kind), pr["mu"], pr["lam"], pr["rho"]))
    return ds


def _batch(probs, kind, prec=0):
    import paper_2104_13466_gb300 as s
    return s.Batch(probs, kind, precision=prec)


def _random_state(b, ds, scale, seed):
    u = np.zeros(b.total)
    for i, d in enumerate(ds):
        h = min(d.mesh.h) / d.mesh.P
        u[b.offsets[i]:b.offsets[i] + b.ndofs[i]] = random_vector(b.ndofs[i], seed + i, scale * h)
    return u


@pytest.mark.parametrize("kind", ["sdme_h", "nodal"])
def test_batch_internal_force_and_tangent_fp64(kind):
    probs = _problems()
    b = _batch(probs, kind)
    ds = _oracles(probs, kind)
    assert [d.mesh.ndof for d in ds] == b.ndofs
    u = _random_state(b, ds, 0.05, 10)
    x = random_vector(b.total, 3)
    R = b.zeros()
    b.internal_force(_dev(u), R)
    y = b.zeros()
    b.tangent_apply(_dev(u), 40.0, _dev(x), y)
    Rh, yh = _host(R), _host(y)
    for i, d in enumerate(ds):
        seg = slice(b.offsets[i], b.offsets[i] + b.ndofs[i])
        assert _rel(Rh[seg], d.internal_force(u[seg])) < TOL64, i
        assert _rel(yh[seg], d.effective_apply(u[seg], x[seg], b1=40.0)) < TOL64, i
    # padding between segments stays untouched
    pad = np.ones(b.total, dtype=bool)
    for i in range(b.nprob):
        pad[b.offsets[i]:b.offsets[i] + b.ndofs[i]] = False
    assert np.all(Rh[pad] == 0.0)


def test_batch_tangent_mixed():
    import paper_2104_13466_gb300 as s
    probs = _problems(seed=1)
    b = _batch(probs, "sdme_m", prec=s.MIXED_FP32)
    ds = _oracles(probs, "sdme_m")
    u = _random_state(b, ds, 0.05, 20)
    x = random_vector(b.total, 4)
    y = b.zeros()
    b.tangent_apply(_dev(u), 10.0, _dev(x), y)
    yh = _host(y)
    for i, d in enumerate(ds):
        seg = slice(b.offsets[i], b.offsets[i] + b.ndofs[i])
        assert _rel(yh[seg], d.effective_apply(u[seg], x[seg], b1=10.0)) < TOL32, i


# largest tile (elements per work item of the persistent launch) per order:
# min(4, 320 // threads per element)
MAX_TILE = {1: 4, 2: 4, 3: 3, 4: 2, 5: 2, 6: 1, 7: 1, 8: 1}


@pytest.mark.parametrize("persist", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_batch_newmark_steps(prec, persist):
    # persist = 1: the PCG operator as one launch across the order groups,
    # each order at its largest tile (several elements per CTA)
    probs = _problems(seed=2, n=5, orders=(2, 3, 4), max_e=2)
    b = _batch(probs, "sdme_h", prec=prec)
    b.set_persistent(persist, MAX_TILE if persist else None)
    ds = _oracles(probs, "sdme_h")
    mags = [0.05 * pr["mu"] for pr in probs]
    f = b.zeros()
    b.traction_load("zmax", [(0.0, 0.0, -m) for m in mags], f)
    fh = _host(f)
    u, v, a = b.zeros(), b.zeros(), b.zeros()
    states = [(np.zeros(d.mesh.ndof),) * 3 for d in ds]
    dt = 0.01
    for n in range(1, 3):
        stats = b.newmark_step(u, v, a, dt, f * (n / 2.0), newton_tol=1e-12, pcg_rtol=1e-13, mixed_rtol=1e-5)
        assert all(st["converged"] for st in stats)
        for i, d in enumerate(ds):
            seg = slice(b.offsets[i], b.offsets[i] + b.ndofs[i])
            uo, vo, ao = states[i]
            uo, vo, ao, so = solvers.newmark_step(d, uo, vo, ao, fh[seg] * (n / 2.0), dt, tol=1e-12, pcg_rtol=1e-13)
            states[i] = (uo, vo, ao)
    uh, vh, ah = _host(u), _host(v), _host(a)
    for i in range(b.nprob):
        seg = slice(b.offsets[i], b.offsets[i] + b.ndofs[i])
        uo, vo, ao = states[i]
        if prec == 0:
            assert _rel(uh[seg], uo) < 1e-9 and _rel(vh[seg], vo) < 1e-8 and _rel(ah[seg], ao) < 1e-7, i
        else:
            assert _rel(uh[seg], uo) < 1e-8 and _rel(vh[seg], vo) < 1e-6, i
    # each problem keeps its own Newton record
    assert len(stats) == b.nprob and all(st["newton_iters"] >= 1 for st in stats)


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_persistent_high_orders(prec):
    # orders 1, 5 and 8 in one persistent launch (P = 8 fills the CTA, P = 1
    # and 5 share it among 4 and 2 elements), a ragged element count per
    # problem (items end short), against the oracle's Newmark step
    probs = [dict(elems=(2, 1, 1), lengths=(1.0, 0.7, 0.9), clamp={"zmin": (0, 1, 2)}, mu=400.0, lam=600.0,
                  rho=1.0, P=8),
             dict(elems=(3, 1, 2), lengths=(1.0, 0.8, 1.2), clamp={"zmin": (0, 1, 2)}, mu=900.0, lam=1500.0,
                  rho=1.0, P=1),
             dict(elems=(1, 3, 1), lengths=(0.9, 1.0, 0.8), clamp={"zmin": (0, 1, 2)}, mu=300.0, lam=900.0,
                  rho=1.0, P=5)]
    b = _batch(probs, "sdme_h", prec=prec)
    b.set_persistent(1, MAX_TILE)
    ds = _oracles(probs, "sdme_h")
    f = b.zeros()
    b.traction_load("zmax", [(0.0, 0.0, -0.05 * pr["mu"]) for pr in probs], f)
    fh = _host(f)
    u, v, a = b.zeros(), b.zeros(), b.zeros()
    stats = b.newmark_step(u, v, a, 0.01, f, newton_tol=1e-12, pcg_rtol=1e-13, mixed_rtol=1e-5)
    assert all(st["converged"] for st in stats)
    assert b.persistent_info()["on"]
    uh = _host(u)
    z = [np.zeros(d.mesh.ndof) for d in ds]
    for i, d in enumerate(ds):
        seg = slice(b.offsets[i], b.offsets[i] + b.ndofs[i])
        uo, _, _, _ = solvers.newmark_step(d, z[i], z[i], z[i], fh[seg], 0.01, tol=1e-12, linear="direct")
        assert _rel(uh[seg], uo) < (1e-9 if prec == 0 else 1e-8), i


def test_batch_persistent_tiles_validated():
    import paper_2104_13466_gb300 as s
    b = _batch(_problems(n=2), "sdme_h")
    with pytest.raises(s.SdmeError):
        b.set_persistent(1, {8: 2})          # a P = 8 element needs all 320 threads
    with pytest.raises(s.SdmeError):
        b.set_persistent(2)


def test_batch_tuner_keeps_results():
    probs = _problems(seed=3, n=6)
    b = _batch(probs, "sdme_h")
    ds = _oracles(probs, "sdme_h")
    u = _random_state(b, ds, 0.05, 30)
    x = random_vector(b.total, 5)
    y0 = b.zeros()
    b.tangent_apply(_dev(u), 5.0, _dev(x), y0)
    tuned = b.tune(reps=2)
    assert sorted(p for p, _, _ in tuned) == sorted({pr["P"] for pr in probs})
    assert all(ms > 0 for _, _, ms in tuned)
    info = b.persistent_info()
    assert info["persist_ms"] > 0 and info["groups_ms"] > 0
    assert all(1 <= info["kper"][pr["P"]] <= MAX_TILE[pr["P"]] for pr in probs)
    y1 = b.zeros()
    b.tangent_apply(_dev(u), 5.0, _dev(x), y1)
    assert _rel(_host(y1), _host(y0)) < 1e-13


def test_batch_rejects_invalid_problems():
    import paper_2104_13466_gb300 as s
    bad = _problems(n=2)
    bad[1]["P"] = 9
    with pytest.raises(s.SdmeError):
        _batch(bad, "sdme_h")


def test_batch_single_problem_and_idle_problems():
    # one problem alone, and a batch where some problems carry no load: those
    # converge at Newton iteration 0 while the others iterate
    probs = _problems(seed=4, n=4, orders=(2, 3), max_e=2)
    one = _batch(probs[:1], "sdme_h")
    ds = _oracles(probs[:1], "sdme_h")
    u = _random_state(one, ds, 0.05, 40)
    R = one.zeros()
    one.internal_force(_dev(u), R)
    assert _rel(_host(R)[:one.ndofs[0]], ds[0].internal_force(u[:one.ndofs[0]])) < TOL64
    b = _batch(probs, "sdme_m")
    f = b.zeros()
    b.traction_load("zmax", [(0.0, 0.0, -5.0 if i % 2 else 0.0) for i in range(b.nprob)], f)
    u, v, a = b.zeros(), b.zeros(), b.zeros()
    stats = b.newmark_step(u, v, a, 0.01, f, newton_tol=1e-10)
    for i, st in enumerate(stats):
        assert st["converged"]
        if i % 2 == 0:
            assert st["newton_iters"] == 0 and st["pcg_iters_total"] == 0
            assert float(b.segment(u, i).abs().max()) == 0.0
        else:
            assert st["newton_iters"] >= 1


def test_batch_refuses_planar_meshes():
    import paper_2104_13466_gb300 as s
    probs = _problems(n=2)
    probs[0]["elems"] = (2, 2)
    probs[0]["lengths"] = (1.0, 1.0)
    with pytest.raises(s.SdmeError):
        _batch(probs, "sdme_h")
