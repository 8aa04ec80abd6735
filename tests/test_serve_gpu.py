"""GPU tests of the trained-basis file format, the noise-model helper and
the serving path (Sec. 2.6: new spectra are projected on the frozen basis
and reconstructed with its cached coefficients).

Serving runs the same kernels as fkk_apply row by row, so its outputs must
equal fkk_apply's bit for bit, however the tiles are batched.
"""
import threading

import numpy as np
import pytest

import oracle as O
from paper_2005_07132_gb300.synth import CubeSpec, make_cube

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FKK_ERR_TIMEOUT, FKK_ERR_BAD_FILE, FKK_ERR_SHUTDOWN = -4, -6, -7


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


def test_serve_large_host_tile_in_chunks(fk, ctx, trained, tmp_path):
    cube, x, ref, basis = trained
    cache = tmp_path / "tune.txt"
    cache.write_text("max_batch=1000\n")  # staging of 1,000 spectra
    srv = fk.Server(ctx, basis, tune_cache=cache)
    big = torch.cat([x] * 3).contiguous()  # 9,216 spectra
    want = _reference(fk, ctx, basis, big)
    tile = big.cpu().pin_memory()
    out = torch.empty_like(tile).pin_memory()
    rid = srv.submit(tile, out)
    assert srv.wait(rid, 20000) == 0
    assert torch.equal(out.cuda(), want)
    srv.stop()


def test_serve_tune_cache_written(fk, ctx, trained, tmp_path):
    _, _, _, basis = trained
    cache = tmp_path / "fresh.txt"
    srv = fk.Server(ctx, basis, tune_cache=cache)
    srv.stop()
    text = cache.read_text()
    assert text.startswith("max_batch=")
    assert 2048 <= int(text.split("=")[1]) <= 65536


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
