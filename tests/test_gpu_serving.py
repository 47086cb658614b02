"""Serving loop (pint_server_*): requests of different kinds, levels, n_t and
beta admitted by device memory, run concurrently on their own streams, and
each result identical to the same request solved alone."""
import time

import numpy as np
import pytest

from paper_2405_18964_gb300 import binding, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _request(kind, level, K, beta, nu=1e-2, prec=1, seed=0):
    oseen = kind == "oseen"
    x0, x1 = (-1.0, 1.0) if oseen else (0.0, 1.0)
    p = binding.default_params(kind=int(oseen), level=level, n_t=K, tau=1.0 / (K + 1), beta=beta, nu=nu,
                               x0=x0, x1=x1, wind=int(oseen), prec=prec)
    vd = inputs.desired_state(2 ** level, x0, x1, K, 1.0 / (K + 1), 1.0, seed=seed)
    n_blk = 4 * (2 * 2 ** level + 1) ** 2 + 2 * (2 ** level + 1) ** 2
    return p, vd, K * n_blk


# Oseen requests stay on grids where the Uzawa/commutator inner solver works
# (on 16x16 with beta = 1e-2 its inner GMRES stagnates at j = 0)
MIX = [("stokes", 4, 16, 1e-2, 1e-2, 1, 1), ("oseen", 4, 8, 1e-4, 1e-2, 1, 2), ("stokes", 3, 8, 1e-6, 1e-2, 0, 3),
       ("oseen", 3, 16, 1e-3, 2e-2, 1, 4), ("stokes", 5, 4, 1e-4, 1e-2, 1, 5), ("oseen", 5, 4, 1e-2, 2e-2, 0, 6)]


def test_results_same_alone_and_in_the_mix():
    reqs = [_request(*m) for m in MIX]
    alone = []
    srv = binding.Server(max_active=1)
    for p, vd, n in reqs:
        x, info, _, _ = srv.wait(srv.submit(p, vd), n)
        assert info.relres <= 1e-8
        alone.append(x)
    srv.close()
    srv = binding.Server(max_active=4)
    ids = [srv.submit(p, vd) for p, vd, _ in reqs]
    # requests that arrive while others are on the GPU
    extra = [srv.submit(*_request("stokes", 4, 8, 1e-3, seed=20 + k)[:2]) for k in range(3)]
    for k, (rid, (p, vd, n)) in enumerate(zip(ids, reqs)):
        x, info, lat, _ = srv.wait(rid, n)
        assert lat > 0
        assert np.array_equal(x, alone[k]), k
    for rid in extra:
        srv.wait(rid, _request("stokes", 4, 8, 1e-3)[2])
    st = srv.stats()
    assert st["completed"] == len(MIX) + 3 and st["failed"] == 0 and st["active_peak"] > 1
    srv.close()


def test_server_result_equals_direct_solve():
    p, vd, n = _request("oseen", 4, 8, 1e-4, seed=9)
    G = binding.Problem(p)
    G.set_data(vd)
    x_direct = np.zeros(n)
    G.solve_host(x_direct)
    G.close()
    srv = binding.Server(max_active=2)
    x, _, _, _ = srv.wait(srv.submit(p, vd), n)
    srv.close()
    assert np.array_equal(x, x_direct)


def test_admission_by_device_memory():
    reqs = [_request("stokes", 5, 16, 1e-3, seed=k) for k in range(4)]
    est = binding.estimate_device_bytes(reqs[0][0])
    # room for one request at a time: they run one after the other
    srv = binding.Server(max_active=4, device_budget=int(est * 1.5))
    ids = [srv.submit(p, vd) for p, vd, _ in reqs]
    for rid, (_, _, n) in zip(ids, reqs):
        srv.wait(rid, n)
    st = srv.stats()
    assert st["active_peak"] == 1 and st["completed"] == 4 and st["bytes_peak"] <= st["budget_bytes"]
    srv.close()
    # a request larger than the whole budget is refused at submission
    srv = binding.Server(max_active=2, device_budget=int(est // 2))
    with pytest.raises(binding.PintError) as err:
        srv.submit(reqs[0][0], reqs[0][1])
    assert err.value.code == 2
    srv.close()


@pytest.mark.parametrize("kind,level,K,prec", [("stokes", 6, 256, 1), ("stokes", 6, 32, 0), ("oseen", 5, 16, 1),
                                               ("oseen", 3, 4, 0)])
def test_estimate_covers_the_handle(kind, level, K, prec):
    p, _, _ = _request(kind, level, K, 1e-4, prec=prec)
    G = binding.Problem(p)
    actual = G.sizes.device_bytes
    G.close()
    est = binding.estimate_device_bytes(p)
    assert actual <= est <= 1.25 * actual + (80 << 20), (actual, est)


# requests sharing grid, domain, wind, nu and precision: two groups (Stokes
# 16x16, Oseen 32x32) whose members differ in n_t and beta
SHARED = [("stokes", 4, 16, 1e-2, 1e-2, 1, 11), ("stokes", 4, 8, 1e-4, 1e-2, 1, 12),
          ("stokes", 4, 32, 1e-6, 1e-2, 1, 13), ("oseen", 5, 8, 1e-4, 1e-2, 1, 14),
          ("oseen", 5, 16, 1e-5, 1e-2, 1, 15), ("stokes", 4, 16, 1e-3, 1e-2, 1, 16)]


def test_shared_frequency_solves_same_as_alone():
    """share_solves: the frequency solves of the requests on the GPU run in
    shared launches; each result is bit for bit the one of the request
    solved alone, and the batches did hold several requests."""
    reqs = [_request(*m) for m in SHARED]
    alone = []
    for p, vd, n in reqs:
        G = binding.Problem(p)
        G.set_data(vd)
        x = np.zeros(n)
        info = G.solve_host(x)
        G.close()
        assert info.relres <= 1e-8
        alone.append(x)
    srv = binding.Server(max_active=6, share_solves=True)
    try:
        ids = [srv.submit(p, vd) for p, vd, _ in reqs]
        got = [srv.wait(rid, n, check=False) for rid, (_, _, n) in zip(ids, reqs)]
        st = srv.stats()
    finally:
        srv.close()
    for k, (x, info, lat, code) in enumerate(got):
        assert code == 0 and info.relres <= 1e-8, (k, code)
        assert np.array_equal(x, alone[k]), (k, float(np.abs(x - alone[k]).max() / np.abs(alone[k]).max()))
    print(f"shared solves: {st['shared_batches']} batches, {st['shared_member_solves']} member applies, "
          f"largest batch {st['shared_max_members']} requests")
    assert st["completed"] == len(SHARED) and st["failed"] == 0
    assert st["shared_max_members"] >= 2 and st["shared_member_solves"] > st["shared_batches"]
