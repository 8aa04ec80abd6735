"""GPU tests of the trained-basis file format, the noise-model helper and
the serving path (Sec. 2.6: new spectra are projected on the frozen basis
and reconstructed with its cached coefficients).

Serving runs the same kernels as fkk_apply row by row, so its outputs must
equal fkk_apply's bit for bit, however the tiles are batched and whichever
slot runs them; batches in different slots overlap on the device; the HBM
budget bounds each slot's staging, so a host tile larger than a slot is
refused with FKK_ERR_BUDGET and requests that find every slot busy wait.
"""
import threading

import numpy as np
import pytest

import oracle as O
from paper_2005_07132_gb300.synth import CubeSpec, make_cube

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FKK_ERR_BUDGET, FKK_ERR_TIMEOUT, FKK_ERR_BAD_FILE, FKK_ERR_SHUTDOWN = -2, -4, -6, -7


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


@pytest.fixture(scope="module")
def trained(fk, ctx):
    cube = make_cube(CubeSpec(height=48, width=64, n_channels=384, n_species=6, seed=77))
    x = torch.from_numpy(cube.i_cars).cuda()
    ref = torch.from_numpy(cube.i_ref).cuda()
    basis, _, _ = fk.fkk_fit_basis(ctx, x, ref, fk.fit_params(k=16))
    yield cube, x, ref, basis
    basis.close()


def _reference(fk, ctx, basis, tile):
    out = fk.fkk_apply(ctx, basis, tile)
    torch.cuda.synchronize()
    return out


def test_basis_save_load_roundtrip(fk, ctx, trained, tmp_path):
    cube, x, ref, basis = trained
    path = tmp_path / "basis.fkk"
    basis.save(path)
    b2 = fk.fkk_basis_load(ctx, path)
    assert b2.info() == basis.info()
    for art in ("s", "lambda", "v", "f", "b", "h_b", "phi_pec", "h_phi", "v_sec", "c_amp", "c_ph", "q", "energy"):
        np.testing.assert_array_equal(b2.get(art), basis.get(art))
    a1 = _reference(fk, ctx, basis, x)
    a2 = _reference(fk, ctx, b2, x)
    assert torch.equal(a1, a2)
    b2.close()


def test_basis_load_rejects_bad_files(fk, ctx, trained, tmp_path):
    _, _, _, basis = trained
    good = tmp_path / "good.fkk"
    basis.save(good)
    raw = good.read_bytes()
    cases = {
        "flipped": raw[:-100] + bytes([raw[-100] ^ 0x40]) + raw[-99:],
        "truncated": raw[: len(raw) // 2],
        "magic": b"NOTBASIS" + raw[8:],
        "empty": b"",
    }
    for name, data in cases.items():
        p = tmp_path / f"{name}.fkk"
        p.write_bytes(data)
        with pytest.raises(fk.FkkError) as e:
            fk.fkk_basis_load(ctx, p)
        assert e.value.status == FKK_ERR_BAD_FILE, name
    with pytest.raises(fk.FkkError) as e:
        fk.fkk_basis_load(ctx, tmp_path / "missing.fkk")
    assert e.value.status == FKK_ERR_BAD_FILE


def test_noise_scale_matches_oracle(fk, ctx):
    r = np.random.default_rng(3)
    mean = r.uniform(0.5, 40.0, 300).astype(np.float32)
    f = fk.fkk_noise_scale(ctx, torch.from_numpy(mean).cuda(), 0.7, 1.3).cpu().numpy()
    np.testing.assert_allclose(f, O.noise_scale(mean.astype(np.float64), 0.7, 1.3), rtol=1e-13)
    with pytest.raises(fk.FkkError):
        fk.fkk_noise_scale(ctx, torch.from_numpy(mean).cuda(), 0.0, 0.0)


def test_serve_device_and_host_tiles_equal_apply(fk, ctx, trained, tmp_path):
    cube, x, ref, basis = trained
    n, m = x.shape
    want = _reference(fk, ctx, basis, x)
    srv = fk.Server(ctx, basis)
    # device tiles of mixed sizes (batched together), pinned host tiles, and
    # one tile larger than the staging buffers
    cuts = [0, 1, 7, 300, 301, 1024, 2000, n]
    ids, outs = [], []
    for a, b in zip(cuts[:-1], cuts[1:]):
        if (a // 7) % 2 == 0:
            tile = x[a:b].contiguous()
            out = torch.full((b - a, m), float("nan"), device="cuda")
        else:
            tile = x[a:b].cpu().pin_memory()
            out = torch.full((b - a, m), float("nan")).pin_memory()
        ids.append(srv.submit(tile, out))
        outs.append((a, b, out))
    for rid in ids:
        assert srv.wait(rid, 20000) == 0
    for a, b, out in outs:
        assert torch.equal(out.cuda(), want[a:b])
    st = srv.stats()
    assert 0 < st["p50_ms"] <= st["p99_ms"] and st["spectra_per_s"] > 0
    srv.stop()


def _pinned(t):
    return t.cpu().pin_memory()


def test_serve_budget_defers_then_completes_and_refuses(fk, trained):
    """A context budget of three slots of 4,096 spectra: a host tile of
    5,000 can never be staged (FKK_ERR_BUDGET at submit); four tiles of 3,000
    (no two fit one slot) take the three slots and the fourth waits for one
    to free, then completes with the same output as fkk_apply."""
    cube, x, ref, basis = trained
    m = x.shape[1]
    small = fk.Context(0, hbm_budget_bytes=3 * 2 * 4096 * m * 4 + (1 << 20))
    srv = fk.Server(small, basis)
    big = _pinned(torch.cat([x, x])[:5000].contiguous())
    with pytest.raises(fk.FkkError) as e:
        srv.submit(big, torch.empty_like(big).pin_memory())
    assert e.value.status == FKK_ERR_BUDGET
    tiles = [_pinned(torch.cat([x, x])[i * 700:i * 700 + 3000].contiguous()) for i in range(4)]
    outs = [torch.empty_like(t).pin_memory() for t in tiles]
    ids = [srv.submit(t, o) for t, o in zip(tiles, outs)]
    for rid in ids:
        assert srv.wait(rid, 20000) == 0
    for t, o in zip(tiles, outs):
        assert torch.equal(o.cuda(), _reference(fk, small, basis, t.cuda()))
    log = srv.batch_log()
    assert len(log) == 4 and np.all(log[:, 3] == 1) and np.all(log[:, 4] == 3000)
    # the fourth batch was admitted only after one of the first three ended
    assert log[3, 0] >= log[:3, 1].min()
    srv.stop()
    small.close()


def test_serve_batches_overlap_and_equal_alone(fk, ctx, trained):
    """Host tiles submitted together run as batches in different slots whose
    event intervals intersect on the device; each result equals the tile's
    own fkk_apply bit for bit."""
    cube, x, ref, basis = trained
    big = torch.cat([x] * 8).contiguous()  # 24,576 spectra per tile
    tiles = [_pinned(torch.roll(big, i * 37, 0)) for i in range(9)]
    outs = [torch.empty_like(t).pin_memory() for t in tiles]
    srv = fk.Server(ctx, basis)
    ids = [srv.submit(t, o) for t, o in zip(tiles, outs)]
    for rid in ids:
        assert srv.wait(rid, 30000) == 0
    log = srv.batch_log()
    assert len(log) >= 2
    overlaps = sum(1 for i in range(len(log)) for j in range(i + 1, len(log))
                   if log[i, 2] != log[j, 2] and log[i, 0] < log[j, 1] and log[j, 0] < log[i, 1])
    assert overlaps >= 1, log
    for t, o in zip(tiles, outs):
        assert torch.equal(o.cuda(), _reference(fk, ctx, basis, t.cuda()))
    srv.stop()


def test_serve_tune_cache_written_and_read(fk, ctx, trained, tmp_path):
    _, x, _, basis = trained
    cache = tmp_path / "fresh.txt"
    srv = fk.Server(ctx, basis, tune_cache=cache)
    srv.stop()
    text = cache.read_text()
    vals = dict(line.split("=") for line in text.split())
    assert 2048 <= int(vals["max_batch"]) <= 65536 and int(vals["stages"]) in (2, 3, 4)
    # a cached max_batch bounds the slots: a host tile above it is refused
    cache.write_text("max_batch=1024\nstages=2\n")
    srv = fk.Server(ctx, basis, tune_cache=cache)
    tile = _pinned(x[:1100].contiguous())
    with pytest.raises(fk.FkkError) as e:
        srv.submit(tile, torch.empty_like(tile).pin_memory())
    assert e.value.status == FKK_ERR_BUDGET
    ok = _pinned(x[:1024].contiguous())
    out = torch.empty_like(ok).pin_memory()
    assert srv.wait(srv.submit(ok, out), 20000) == 0
    assert torch.equal(out.cuda(), _reference(fk, ctx, basis, ok.cuda()))
    srv.stop()


def test_serve_wait_timeout_then_complete(fk, ctx, trained):
    cube, x, ref, basis = trained
    srv = fk.Server(ctx, basis)
    big = torch.cat([x] * 40).contiguous()  # ~123k spectra per tile
    outs = [torch.empty_like(big) for _ in range(12)]
    small = x[:64].contiguous()
    out_small = torch.empty_like(small)
    rs = [srv.submit(big, o) for o in outs]  # milliseconds of work queued ahead
    r2 = srv.submit(small, out_small)
    assert srv.wait(r2, 0) == FKK_ERR_TIMEOUT
    for r in rs:
        assert srv.wait(r, -1) == 0
    assert srv.wait(r2, -1) == 0
    assert srv.wait(r2, 0) != 0  # released id
    srv.stop()


def test_serve_stop_cancels_queued(fk, ctx, trained):
    """Queued requests end with FKK_ERR_SHUTDOWN and a thread blocked in
    wait returns; the waiter is inside wait before stop is called (the
    queue holds tens of milliseconds of work)."""
    import time

    cube, x, ref, basis = trained
    srv = fk.Server(ctx, basis)
    big = torch.cat([x] * 20).contiguous()  # ~61k spectra per tile
    out_big = torch.empty_like(big)
    ids = [srv.submit(big, out_big) for _ in range(400)]  # ~0.1 s of work
    got = {}

    def waiter():
        got["last"] = srv.wait(ids[-1], -1)

    th = threading.Thread(target=waiter)
    th.start()
    time.sleep(0.01)
    srv.stop()
    th.join(timeout=30)
    assert not th.is_alive()
    assert got["last"] == FKK_ERR_SHUTDOWN
    # the server is gone: new submissions are impossible through this object
    with pytest.raises(Exception):
        srv.submit(big, out_big)
