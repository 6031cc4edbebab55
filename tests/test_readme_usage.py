"""The usage example of the package overview, run as written on small data (GPU)."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_readme_usage(gbaes):
    rng = np.random.default_rng(77)
    k = gbaes.Key(bytes(32))  # AES-256
    x = torch.randint(0, 256, (1 << 20,), dtype=torch.uint8, device="cuda")
    c = gbaes.encrypt_ecb(k, x)
    assert torch.equal(gbaes.decrypt_ecb(k, c), x)

    raw_keys = [rng.integers(0, 256, b // 8, dtype=np.uint8).tobytes() for b in (128, 192, 256, 128)]
    keys = [gbaes.Key(r) for r in raw_keys]
    nbytes = np.array([16, 4096, 1 << 16, 48])
    in_off = np.concatenate([[0], np.cumsum(nbytes)[:-1]])
    out_off = in_off.copy()
    key_index = np.arange(4)
    decrypt = np.array([0, 1, 0, 1])
    d = gbaes.make_descs(in_off, out_off, nbytes // 16, key_index, decrypt)
    plan = gbaes.BatchPlan(d, keys)
    xb = x[: int(nbytes.sum())]
    y = torch.empty_like(xb)
    plan.launch(xb, y)
    xs, ys = xb.cpu().numpy(), y.cpu().numpy()
    for i in range(4):
        a, n = int(in_off[i]), int(nbytes[i])
        assert np.array_equal(ys[a:a + n], oracle.ecb(raw_keys[i], len(raw_keys[i]) * 8, xs[a:a + n],
                                                       decrypt=bool(decrypt[i])))

    torch.cuda.synchronize()
    srv = gbaes.Server(keys, resident=True)
    z = torch.zeros_like(xb)
    srv.submit(7, 2, xb.data_ptr(), z.data_ptr(), 4096 // 16, decrypt=False)
    srv.drain(1.0)
    done = srv.poll_all()
    srv.close()
    assert done["id"].tolist() == [7] and done["status"][0] == 0
    assert np.array_equal(z[:4096].cpu().numpy(), oracle.ecb(raw_keys[2], 256, xs[:4096]))

    host_in = torch.from_numpy(xs.copy()).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    want = oracle.ecb(raw_keys[0], 128, xs)
    for mode in (gbaes.PIPE_DIRECT, gbaes.PIPE_STAGED):
        host_out.zero_()
        gbaes.Pipeline(mode=mode).ecb(keys[0], host_in, host_out)
        torch.cuda.synchronize()
        assert np.array_equal(host_out.numpy(), want)
    host_out.zero_()
    gbaes.ecb_ex(keys[0], host_in, host_out)
    torch.cuda.synchronize()
    assert np.array_equal(host_out.numpy(), want)
