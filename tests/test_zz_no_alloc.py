"""helm_dot_noalloc, the dot product for callers that cannot allocate device
memory (graph capture that forbids allocation, real-time loops, hosts with
their own memory manager): its scratch is a fixed array inside the library.
It must give the result of helm_dot bit for bit (each thread adds the same
elements in the same order, and the block partials are added in block
order), for complex128 and complex64 inputs, on consecutive calls that share
that array, and lie within the dot-product tolerance of the other GPU tests
(1e-13 * sum |x_i| |y_i|, complex64: 1e-6) of the FP64 value.  This file is collected last, so a stop-at-first-failure run has
already run every other test."""
import ctypes

import numpy as np
import pytest

import helmgen as g

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2112_11880_gb300 as helm  # noqa: E402

DEV = torch.device("cuda:0")


def _c_abi_dot(fn, x, y, out, conj, stream):
    """Call a dot entry point through the C ABI (ctypes, raw pointers)."""
    st = fn(ctypes.c_int64(x.numel()), helm.HELM_C128 if x.dtype == torch.complex128 else helm.HELM_C64,
            ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), 1 if conj else 0,
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    assert st == helm.HELM_OK, helm.STATUS_NAMES.get(st, st)


@pytest.mark.parametrize("n,conj,dtype", [(1_000_003, True, torch.complex128), (257, False, torch.complex128),
                                          (1_000_003, True, torch.complex64)])
def test_dot_noalloc_matches_dot_on_two_calls(n, conj, dtype):
    from paper_2112_11880_gb300 import build
    build.build()
    lib = helm.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    pairs = [(g.complex_vector(n, 31), g.complex_vector(n, 32)),
             (g.complex_vector(n, 33), 2.5 * g.complex_vector(n, 34))]
    for xh, yh in pairs:          # two calls in a row share the scratch array
        x = torch.as_tensor(xh, device=DEV).to(dtype)
        y = torch.as_tensor(yh, device=DEV).to(dtype)
        ref = torch.zeros(1, dtype=torch.complex128, device=DEV)
        out = torch.full((1,), complex("nan+nanj"), dtype=torch.complex128, device=DEV)
        _c_abi_dot(lib.helm_dot, x, y, ref, conj, stream)
        _c_abi_dot(lib.helm_dot_noalloc, x, y, out, conj, stream)
        torch.cuda.synchronize()
        assert torch.equal(torch.view_as_real(out), torch.view_as_real(ref))
        d = complex(out.cpu().numpy()[0])
        xe = x.cpu().numpy().astype(np.complex128)
        ye = y.cpu().numpy().astype(np.complex128)
        exact = np.vdot(xe, ye) if conj else np.dot(xe, ye)
        tol = 1e-13 if dtype == torch.complex128 else 1e-6
        assert abs(d - exact) <= tol * float(np.sum(np.abs(xe) * np.abs(ye)))


def test_dot_noalloc_rejects_sizes_beyond_the_maximum():
    lib = helm.load_library()
    out = torch.zeros(1, dtype=torch.complex128, device=DEV)
    x = torch.zeros(4, dtype=torch.complex128, device=DEV)
    st = lib.helm_dot_noalloc(ctypes.c_int64(1 << 31), helm.HELM_C128, ctypes.c_void_p(x.data_ptr()),
                              ctypes.c_void_p(x.data_ptr()), 1, ctypes.c_void_p(out.data_ptr()), None)
    assert st == helm.HELM_ERR_INVALID
