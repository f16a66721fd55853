"""dirac_apply_static: the canonical apply without device allocation.

It is for callers that cannot allocate device memory while they run (a
stream being captured into a CUDA graph, loops that must not trigger the
device synchronisation of cudaMalloc / cudaFree, hosts whose device memory
is all reserved by their own allocator).  Its work fields live in a fixed
array of the library's device image.  This file runs last so that a failure
here does not hide the results of the other GPU tests."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1808_05506_gb300 as dg
    torch.cuda.set_device(0)
    return dg


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("op,mass", [("wilson", 0.124), ("staggered", 0.05), ("brillouin", 0.05)])
def test_static_apply_matches_apply_twice(dg, op, mass):
    L, Nv = (8, 8, 4, 8), 3
    ns = 1 if op == "staggered" else 4
    V = synth.round_to(synth.gauge_links(L, 3, "near_identity", 500), "f32")
    psi = synth.round_to(synth.spinor(L, Nv, ns, 3, 501), "f32")
    D = dg.Dirac(op, L, Nv, mass, "f32")
    D.set_links(torch.from_numpy(V.astype(np.complex64)).cuda())
    x = torch.from_numpy(psi.astype(np.complex64)).cuda()
    for dagger in (0, 1):
        ref = D.apply(x, dagger=bool(dagger))            # the allocating entry point
        for call in range(2):                             # two calls in a row share the array
            y = torch.full_like(x, float("nan"))
            st = dg.dirac_apply_static(D.h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()), dagger)
            assert st == dg.OK, dg.last_error(D.h)
            torch.cuda.synchronize()
            assert _rel(y, ref) <= 1e-6, (dagger, call)
    D.close()


def test_static_apply_rejects_too_large(dg):
    L, Nv = (16, 16, 16, 16), 8                           # 2 x 50 MB of work fields > 64 MiB
    D = dg.Dirac("wilson", L, Nv, 0.12, "f32")
    D.set_links(torch.from_numpy(synth.gauge_links(L, 3, "unit", 0).astype(np.complex64)).cuda())
    x = D.new_canonical()
    y = D.new_canonical()
    st = dg.dirac_apply_static(D.h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()), 0)
    assert st == dg.ERR_INVALID_ARG
    assert "static area holds" in dg.last_error(D.h)
    D.close()
