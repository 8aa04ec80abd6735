"""The device-side timeout path, exercised without faulting or hanging the
GPU: fkk_test_stall_next_eigensolve makes the next tridiagonal reduction wait,
in its first column exchange, for a tag that no step publishes, with a short
bound.  The bounded wait runs out, the kernel records FKK_ERR_TIMEOUT and
returns; fkk_sync_status reports it, and the context stays usable."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FKK_ERR_TIMEOUT = -4


@pytest.fixture(scope="module")
def fk():
    from paper_2005_07132_gb300 import build
    build.build()
    import paper_2005_07132_gb300 as m
    return m


def _spd(m, seed):
    r = np.random.default_rng(seed)
    B = r.standard_normal((2 * m, m))
    return B.T @ B


def test_eigensolve_wait_runs_out_then_context_recovers(fk):
    ctx = fk.Context(0)
    G = _spd(300, 1)
    g = torch.from_numpy(G).cuda()
    assert ctx.sync_status()[0] == 0
    ctx.stall_next_eigensolve()
    t0 = time.perf_counter()
    fk.fkk_eig_topk(ctx, g, 8)
    st, _ = ctx.sync_status()
    elapsed = time.perf_counter() - t0
    assert st == FKK_ERR_TIMEOUT
    assert elapsed < 10.0  # the bound, not a hang
    # one-shot: the next eigensolve on the same context completes and is right
    lam, V = fk.fkk_eig_topk(ctx, g, 8)
    assert ctx.sync_status()[0] == 0
    w = np.linalg.eigvalsh(G)[::-1]
    lam = lam.cpu().numpy()
    V = V.cpu().numpy()
    assert np.abs(lam - w[:8]).max() <= 1e-12 * w[0]
    assert np.linalg.norm(G @ V - V * lam) <= 1e-12 * np.linalg.norm(G)
    ctx.close()


def test_fit_after_a_timed_out_fit(fk):
    """A fit whose eigensolve timed out reports it; the next fit on the same
    context is the same as on a fresh one, bit for bit."""
    from paper_2005_07132_gb300.synth import CubeSpec, make_cube
    cube = make_cube(CubeSpec(24, 24, 200, 5, "gauss", 50.0, seed=31))
    x = torch.from_numpy(cube.i_cars).cuda()
    ref = torch.from_numpy(cube.i_ref).cuda()
    ctx = fk.Context(0)
    ctx.stall_next_eigensolve()
    b0, _, _ = fk.fkk_fit_basis(ctx, x, ref, fk.fit_params(k=6))
    assert ctx.sync_status()[0] == FKK_ERR_TIMEOUT
    b0.close()
    b1, im1, _ = fk.fkk_fit_basis(ctx, x, ref, fk.fit_params(k=6))
    assert ctx.sync_status()[0] == 0
    fresh = fk.Context(0)
    b2, im2, _ = fk.fkk_fit_basis(fresh, x, ref, fk.fit_params(k=6))
    torch.cuda.synchronize()
    assert torch.equal(im1, im2)
    for b in (b1, b2):
        b.close()
    ctx.close()
    fresh.close()
