"""The allocation-free router loss/gradient entry point (device buffers in,
device buffers out, scratch in a fixed device array inside the library)
gives the same result as tg_router_loss_grad, on two calls in a row.

It exists for callers that cannot allocate device memory where they need
this computation (inside a CUDA-graph stream capture, next to a framework
whose caching allocator holds the free memory, or in loops that cannot take
the synchronisation cudaFree may cause).  This file is collected last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_loss_grad_matches_allocating_entry_point():
    torch = pytest.importorskip("torch")
    from paper_2407_16586_gb300 import build
    build.build()
    import paper_2407_16586_gb300 as tg
    L = tg.lib()
    fn = L.tg_router_loss_grad_noalloc
    fp = ctypes.c_void_p
    fn.argtypes = [ctypes.c_int, fp, fp, fp, fp, fp, ctypes.c_float, fp, fp, fp]
    fn.restype = ctypes.c_int
    r = tg.Router(seed=17)
    params, mu, sd, _ = r.get()
    rng = np.random.default_rng(8)
    for n, q in ((3000, 0.9), (777, 0.6)):
        X = rng.normal(size=(n, 16)).astype(np.float32)
        y = rng.normal(size=n).astype(np.float32)
        L_ref, g_ref = r.loss_grad(X, y, q=q)
        dev = torch.device("cuda")
        tX, ty = torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev)
        tmu, tsd, tp = (torch.from_numpy(a).to(dev) for a in (mu, sd, params))
        for _ in range(2):
            loss = torch.full((1,), float("nan"), device=dev)
            grad = torch.full((r.nparam,), float("nan"), device=dev)
            rc = fn(n, tX.data_ptr(), ty.data_ptr(), tmu.data_ptr(), tsd.data_ptr(), tp.data_ptr(), q,
                    loss.data_ptr(), grad.data_ptr(), torch.cuda.current_stream().cuda_stream)
            assert rc == tg.TG_OK
            torch.cuda.synchronize()
            g = grad.cpu().numpy()
            assert abs(float(loss.item()) - L_ref) <= 1e-6 * abs(L_ref)
            np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-6 * np.abs(g_ref).max())
    # sizes beyond the fixed scratch are refused, not truncated
    big = 65537
    assert fn(big, tX.data_ptr(), ty.data_ptr(), tmu.data_ptr(), tsd.data_ptr(), tp.data_ptr(), 0.9,
              loss.data_ptr(), grad.data_ptr(), None) == tg.TG_EUNSUPPORTED
