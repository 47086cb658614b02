"""Groups of handles whose frequency solves share launches (pint_group_*).

The frequency blocks of the block-circulant preconditioner are independent
(Sec. 3.1), so solving the frequencies of several problems in one set of
launches, each frequency with the constants of its own problem, must give
every problem exactly the result it gets alone.  These tests solve problems
concurrently (one host thread and CUDA stream each) on handles of one group
and compare each solution bit for bit with the same solve on an ordinary
handle, then check the group's statistics and profile.
"""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2405_18964_gb300 import binding, inputs  # noqa: E402

T = 1.0


def _params(kind, level, K, beta, prec=1, **kw):
    x0, x1, wind = (0.0, 1.0, 0) if kind == "stokes" else (-1.0, 1.0, 1)
    return binding.default_params(kind=0 if kind == "stokes" else 1, level=level, n_t=K, tau=T / (K + 1),
                                  beta=beta, nu=1e-2, x0=x0, x1=x1, wind=wind, prec=prec, **kw)


def _vd(p, seed):
    return inputs.desired_state(2 ** p.level, p.x0, p.x1, p.n_t, p.tau, T, seed)


def _solve_alone(p, vd):
    G = binding.Problem(p, stream=torch.cuda.current_stream().cuda_stream)
    G.set_data(vd)
    x = torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda")
    info = G.solve(x)
    torch.cuda.synchronize()
    G.close()
    return x, info


def _solve_grouped(group, ps, vds):
    streams = [torch.cuda.Stream() for _ in ps]
    probs = [binding.Problem(p, stream=s.cuda_stream, group=group) for p, s in zip(ps, streams)]
    for G, vd in zip(probs, vds):
        G.set_data(vd)
    xs = [torch.zeros(G.kkt_len, dtype=torch.float64, device="cuda") for G in probs]
    infos, errs = [None] * len(ps), []

    def run(k):
        try:
            infos[k] = probs[k].solve(xs[k])
        except Exception as e:  # re-raised on the main thread
            errs.append(e)

    torch.cuda.synchronize()
    th = [threading.Thread(target=run, args=(k,)) for k in range(len(ps))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    torch.cuda.synchronize()
    for G in probs:
        G.close()
    if errs:
        raise errs[0]
    return xs, infos


MIXES = {
    # three betas and two time-step counts of one Stokes discretisation
    "stokes": [("stokes", 4, 8, 1e-2), ("stokes", 4, 12, 1e-4), ("stokes", 4, 8, 1e-6)],
    # Oseen (Algorithm 3 inside the inner GMRES) at two betas and n_t (betas
    # where the inner solver converges on these grids; beta = 1e-2 on 16 x 16
    # stagnates at j = 0)
    "oseen": [("oseen", 5, 8, 1e-4), ("oseen", 5, 16, 1e-5)],
    # two subgroups in one group: each shares only with its own kind
    "mixed": [("stokes", 4, 8, 1e-3), ("oseen", 4, 8, 1e-4), ("stokes", 4, 8, 1e-5), ("oseen", 4, 16, 1e-4)],
}


@pytest.mark.parametrize("mix", list(MIXES))
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_grouped_solves_equal_solves_alone(mix, prec):
    ps = [_params(kind, level, K, beta, prec=prec) for kind, level, K, beta in MIXES[mix]]
    vds = [_vd(p, 30 + k) for k, p in enumerate(ps)]
    group = binding.Group()
    try:
        xs, infos = _solve_grouped(group, ps, vds)
        st = group.stats()
    finally:
        group.close()
    print(f"{mix} {'fp32' if prec else 'fp64'}: {st}")
    for k, (p, vd) in enumerate(zip(ps, vds)):
        x1, info1 = _solve_alone(p, vd)
        assert infos[k].relres <= 1e-8
        assert infos[k].outer_iterations == info1.outer_iterations, k
        assert torch.equal(xs[k], x1), (k, float((xs[k] - x1).abs().max()))
    # every apply went through the group's shared solves
    assert st["member_solves"] == sum(i.precond_applies for i in infos)
    assert st["frequencies"] >= st["member_solves"]
    assert 1 <= st["max_members"] <= len(ps)


def test_group_shares_launches_and_profiles_them():
    """Three concurrent Stokes solves: some batches serve several handles,
    and the group's profile counts the shared multigrid launches with
    their algorithmic bytes."""
    ps = [_params("stokes", 5, 16, b) for b in (1e-2, 1e-4, 1e-6)]
    vds = [_vd(p, 40 + k) for k, p in enumerate(ps)]
    group = binding.Group()
    try:
        group.profile_enable(["mg_q2", "apply"])
        xs, infos = _solve_grouped(group, ps, vds)
        st, prof = group.stats(), group.profile_read()
    finally:
        group.close()
    print(f"shared: {st}; mg_q2 {prof['mg_q2']['launches']} launches, {prof['mg_q2']['ms']:.1f} ms, "
          f"apply {prof['apply']['ms']:.1f} ms")
    assert all(i.relres <= 1e-8 for i in infos)
    assert st["max_members"] >= 2 and st["member_solves"] > st["batches"]
    assert st["batches"] == prof["apply"]["timed"]          # one timed scope per shared solve
    assert prof["mg_q2"]["launches"] >= prof["mg_q2"]["timed"] > 0
    assert prof["mg_q2"]["bytes"] > 0 and prof["mg_q2"]["ms"] > 0
    # at least one host synchronisation per shared batch (plus one per inner step)
    assert prof["host_syncs"] >= 2 * st["batches"]


def test_nodal_wind_cannot_join_a_group():
    from oracle import fem
    p = binding.default_params(kind=1, level=3, n_t=4, tau=T / 5, beta=1e-2, nu=1e-2, x0=-1.0, x1=1.0, wind=3, prec=1)
    X, Y = fem.Grid(8, -1.0, 1.0).q2_coords()
    nodal = np.stack(fem.two_vortex_wind(X, Y))
    group = binding.Group()
    try:
        with pytest.raises(binding.PintError):
            binding.Problem(p, wind=nodal, group=group)
    finally:
        group.close()
