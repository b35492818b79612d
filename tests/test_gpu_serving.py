"""The serving engine (solve requests of mixed sizes admitted to worker slots
under an HBM budget) through the C ABI: each result is the same alone and in
a concurrent mix, admission respects the budget, and the device's synthetic
problems are those of the Philox4x32-10 generator's published definition
(re-implemented here on the host)."""
import numpy as np
import pytest

import oracle as O
from paper_1208_4869_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ccg():
    from paper_1208_4869_gb300 import build as B
    B.build()
    from paper_1208_4869_gb300 import ccg as C
    return C


MIX = [dict(kind="dense", n=256, nrhs=1, seed=11, tol=1e-10),
       dict(kind="dense", n=384, nrhs=3, seed=12, tol=1e-6),
       dict(kind="dense", n=512, nrhs=8, seed=13, tol=1e-10),
       dict(kind="dipole", L=8, tol=1e-8),
       dict(kind="dense", n=128, nrhs=2, seed=14, tol=1e-6),
       dict(kind="dipole", L=12, tol=1e-6),
       dict(kind="dense", n=640, nrhs=1, seed=15, tol=1e-6),
       dict(kind="dense", n=512, nrhs=4, seed=16, tol=1e-10)]


def size_of(r):
    if r["kind"] == "dense":
        return r["n"] * r["nrhs"]
    return 3 * int(W.sphere_occupancy(r["L"]).sum())


def test_same_result_alone_and_in_the_mix(ccg):
    alone = []
    sv = ccg.Server(slots=1)
    for r in MIX:
        t = sv.submit(keep_x=True, **r)
        alone.append(sv.wait(t, size_of(r)))
    sv.close()
    sv = ccg.Server(slots=4)
    tickets = [sv.submit(keep_x=True, **r) for r in MIX]
    mixed = [sv.wait(t, size_of(r)) for t, r in zip(tickets, MIX)]
    slots = {res["slot"] for res, _ in mixed}
    sv.close()
    assert len(slots) > 1                       # the mix really ran on several slots
    for r, (ra, xa), (rm, xm) in zip(MIX, alone, mixed):
        assert ra["status"] == 0 and rm["status"] == 0, (r, ra, rm)
        assert np.array_equal(xa, xm), r
        # every tolerance of the mix is below 1e-5, so every result carries a
        # complex128 residual that certifies it
        assert ra["relres"] <= r["tol"], (r, ra)


def test_budget_admission_serialises(ccg):
    n = 512
    one = 16 * n * n + 8 * n * n + 8 * n * n + 40 * n * 8 * 16 + 64 * n * 16   # the engine's estimate for one request
    sv = ccg.Server(slots=4, budget_bytes=int(one * 1.5))
    ts = [sv.submit(kind="dense", n=n, nrhs=1, seed=20 + i, tol=1e-10) for i in range(4)]
    res = [sv.wait(t)[0] for t in ts]
    sv.close()
    res.sort(key=lambda d: d["t_start"])
    for a, b in zip(res, res[1:]):
        assert b["t_start"] >= a["t_done"] - 1e-6
    sv = ccg.Server(slots=4)
    ts = [sv.submit(kind="dense", n=2048, nrhs=1, seed=20 + i, tol=1e-10) for i in range(4)]
    res = sorted((sv.wait(t)[0] for t in ts), key=lambda d: d["t_start"])
    sv.close()
    assert len({r["slot"] for r in res}) > 1
    assert any(b["t_start"] < a["t_done"] for a, b in zip(res, res[1:]))   # overlap when the budget allows


# ---- host restatement of Philox4x32-10 and the engine's normal draws -------
M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85


def philox(c0, c1, c2, c3, k0, k1):
    c = [np.asarray(v, dtype=np.uint64) for v in (c0, c1, c2, c3)]
    k0, k1 = np.uint64(k0), np.uint64(k1)
    mask = np.uint64(0xFFFFFFFF)
    for r in range(10):
        if r:
            k0, k1 = (k0 + np.uint64(W0)) & mask, (k1 + np.uint64(W1)) & mask
        p0, p1 = np.uint64(M0) * c[0], np.uint64(M1) * c[2]
        hi0, lo0, hi1, lo1 = p0 >> np.uint64(32), p0 & mask, p1 >> np.uint64(32), p1 & mask
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


def complex_normal(seed, stream, count):
    idx = np.arange(count, dtype=np.uint64)
    r = philox(idx & np.uint64(0xFFFFFFFF), idx >> np.uint64(32), np.full(count, stream, np.uint64),
               np.zeros(count, np.uint64), seed & 0xFFFFFFFF, seed >> 32)
    u1 = (((r[0] << np.uint64(21)) ^ (r[1] >> np.uint64(11))).astype(np.float64) + 0.5) / 2.0 ** 53
    u2 = (((r[2] << np.uint64(21)) ^ (r[3] >> np.uint64(11))).astype(np.float64) + 0.5) / 2.0 ** 53
    rad = np.sqrt(-np.log(u1))
    return rad * np.cos(2 * np.pi * u2) + 1j * rad * np.sin(2 * np.pi * u2)


def test_generated_problem_matches_host_philox(ccg):
    n, k, seed, shift = 96, 3, 123456789012, 3.0
    A = complex_normal(seed, 0, n * n).reshape(n, n) / np.sqrt(n)
    A[np.diag_indices(n)] += shift + 0.5 + 0.5j
    Y = complex_normal(seed, 1, n * k).reshape(k, n).T          # column-major n x k
    off = (A * np.sqrt(n))[~np.eye(n, dtype=bool)]
    assert abs(np.var(off.real) - 0.5) < 0.05 and abs(np.var(off.imag) - 0.5) < 0.05   # N(0, 1/2) parts
    sv = ccg.Server(slots=1)
    res, x = sv.wait(sv.submit(kind="dense", n=n, nrhs=k, shift=shift, seed=seed, tol=1e-10, keep_x=True), n * k)
    sv.close()
    X = x.reshape(k, n).T
    rel = np.linalg.norm(Y - A @ X, axis=0) / np.linalg.norm(Y, axis=0)
    assert res["status"] == 0 and np.all(rel <= 1e-10), rel
    ref = O.solve(O.DenseOp(np.ascontiguousarray(A)), "bicgstab", np.ascontiguousarray(Y[:, 0]), tol=1e-12,
                  maxit=200)
    assert np.linalg.norm(X[:, 0] - ref.x) / np.linalg.norm(ref.x) < 1e-9


def test_concurrent_operator_creation_under_load(ccg):
    """Sixteen slots that create dipole operators of several sizes at the same
    time, on non-blocking streams, while dense requests load the GPU: every
    mixed-precision dipole request converges and equals its result from a
    single slot (operator uploads must be ordered with the slot's stream)."""
    reqs = []
    for i in range(32):
        reqs.append(dict(kind="dipole", L=[16, 24, 32, 48][i % 4], tol=1e-10))
        reqs.append(dict(kind="dense", n=1024 + 256 * (i % 4), nrhs=1 + i % 8, seed=100 + i, tol=1e-10))
    sv = ccg.Server(slots=16)
    tickets = [sv.submit(keep_x=True, **r) for r in reqs]
    got = [sv.wait(t, size_of(r)) for t, r in zip(tickets, reqs)]
    sv.close()
    alone = {}
    sv = ccg.Server(slots=1)
    for L in (16, 24, 32, 48):
        r = dict(kind="dipole", L=L, tol=1e-10)
        alone[L] = sv.wait(sv.submit(keep_x=True, **r), size_of(r))
    sv.close()
    for r, (res, x) in zip(reqs, got):
        assert res["status"] == 0 and res["relres"] <= 3e-10, (r, res)
        if r["kind"] == "dipole":
            assert np.array_equal(x, alone[r["L"]][1]), r


def test_budget_charges_cached_operators(ccg):
    """A dipole request's operators stay cached on its slot and stay charged
    to the budget until the server is destroyed; a second request of the same
    lattice on that slot adds nothing.  The device memory a request adds
    (after a first request has loaded the kernels and sized the slot's
    workspace) is within its estimate."""
    sv = ccg.Server(slots=1)
    assert sv.charged() == 0
    res, _ = sv.wait(sv.submit(kind="dipole", L=16, tol=1e-10))     # loads the kernels
    assert res["status"] == 0
    charged0 = sv.charged()
    assert charged0 > 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    req = dict(kind="dipole", L=32, tol=1e-10)
    est = ccg.server_estimate(**req)
    res, _ = sv.wait(sv.submit(**req))
    assert res["status"] == 0 and res["relres"] <= 1e-10
    cached = sv.charged() - charged0
    assert 0 < cached < est
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 <= est, (free0 - free1, est)
    res, _ = sv.wait(sv.submit(**req))
    assert res["status"] == 0 and sv.charged() - charged0 == cached
    sv.close()


def test_batching_small_dense_requests(ccg):
    """Small single-right-hand-side dense requests waiting together are solved
    in one many-system launch per step (the 3-column one on the per-slot block
    solver): every result certifies its tolerance, and each request's solution
    is bitwise the same in a batch as alone (a batch of one)."""
    reqs = [dict(kind="dense", n=n, nrhs=k, seed=50 + i, tol=tol)
            for i, (n, k, tol) in enumerate([(512, 1, 1e-10), (1024, 1, 1e-6), (768, 3, 1e-10), (2048, 1, 1e-6),
                                             (600, 1, 1e-10), (1536, 1, 1e-10)])]
    alone = []
    sv = ccg.Server(slots=1)
    for r in reqs:
        alone.append(sv.wait(sv.submit(keep_x=True, **r), size_of(r)))
    sv.close()
    sv = ccg.Server(slots=1)
    # hold the slot with a dipole request so that the dense ones queue up together
    t0 = sv.submit(kind="dipole", L=24, tol=1e-10)
    tickets = [sv.submit(keep_x=True, **r) for r in reqs]
    together = [sv.wait(t, size_of(r)) for t, r in zip(tickets, reqs)]
    sv.wait(t0)
    sv.close()
    starts = {res["t_start"] for res, _ in together}
    assert len(starts) < len(reqs)            # some requests shared a launch
    for r, (ra, xa), (rb, xb) in zip(reqs, alone, together):
        assert ra["status"] == 0 and rb["status"] == 0, (r, ra, rb)
        assert ra["relres"] <= r["tol"] and rb["relres"] <= r["tol"]
        assert np.array_equal(xa, xb), r
