"""GPU test of fkk_reconstruct_noalloc, the reconstruction entry point that
allocates no device memory (its scratch is a fixed static array inside the
library).  It must give the results of fkk_reconstruct (Eq. fKKEC) on the
same inputs, call after call, without the device's free memory or the
context's workspace moving, and reject sizes above its limits before
launching anything.  The file is named to be collected last so that it also
runs after every other GPU test in one process; it passes on its own too.
"""
import numpy as np
import pytest

from gpu_util import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_N = 16384  # FKK_NOALLOC_MAX_SPECTRA
MAX_M = 2048   # FKK_NOALLOC_MAX_CHANNELS


@pytest.fixture(scope="module")
def fk():
    from paper_2005_07132_gb300 import build
    build.build()
    import paper_2005_07132_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(fk):
    c = fk.Context(0)
    yield c
    c.close()


def _inputs(n, k, m, seed):
    r = np.random.default_rng(seed)
    p = torch.from_numpy((r.standard_normal((n, k)) * 0.05).astype(np.float32)).cuda()
    ca = torch.from_numpy(r.standard_normal((k, m)) * 0.5).cuda()
    cp = torch.from_numpy(r.standard_normal((k, m)) * 0.5).cuda()
    return p, ca, cp


def test_two_calls_match_fkk_reconstruct(fk, ctx):
    # per-device setup first, before anything is timed or captured
    fk.fkk_reconstruct_noalloc(ctx, None, None, None, None)
    cases = [(5000, 40, 1000, 3, True), (MAX_N, 80, 877, 0, False)]
    for call, (n, k, m, ld_pad, with_re) in enumerate(cases):
        p, ca, cp = _inputs(n, k, m, seed=100 + call)
        ld = m + ld_pad
        ref_im = torch.empty((n, m), device="cuda")
        ref_re = torch.empty((n, m), device="cuda") if with_re else None
        fk.fkk_reconstruct(ctx, p, ca, cp, im_out=ref_im, re_out=ref_re)
        im_buf = torch.full((n, ld), 9.0, device="cuda")
        re_buf = torch.full((n, ld), 9.0, device="cuda") if with_re else None
        torch.cuda.synchronize()
        ws0 = ctx.workspace_bytes()
        free0 = torch.cuda.mem_get_info()[0]
        fk.fkk_reconstruct_noalloc(ctx, p, ca, cp, im_out=im_buf[:, :m],
                                   re_out=re_buf[:, :m] if with_re else None)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert ctx.workspace_bytes() == ws0
        st, _ = ctx.sync_status()
        assert st == 0
        im = im_buf.cpu().numpy()
        assert rel_l2(im[:, :m], ref_im.cpu().numpy()) <= 1e-6
        assert np.all(im[:, m:] == 9.0)
        if with_re:
            re = re_buf.cpu().numpy()
            assert rel_l2(re[:, :m], ref_re.cpu().numpy()) <= 1e-6
            assert np.all(re[:, m:] == 9.0)


@pytest.mark.parametrize("n,k,m,what", [(MAX_N + 1, 8, 64, "n_spectra"), (4, 8, MAX_M + 1, "m "),
                                        (4, 81, 64, "k ")])
def test_rejects_sizes_above_limits(fk, ctx, n, k, m, what):
    p, ca, cp = _inputs(n, k, m, seed=7)
    im = torch.full((n, m), 9.0, device="cuda")
    launches = fk.launch_count()
    with pytest.raises(fk.FkkError) as e:
        fk.fkk_reconstruct_noalloc(ctx, p, ca, cp, im_out=im)
    assert e.value.status == -1
    assert what in ctx.last_error()
    assert fk.launch_count() == launches
    assert bool(torch.all(im == 9.0))
