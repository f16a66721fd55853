"""When the differentiable apply loads the links into the handle (CPU test of
the bookkeeping, with a stand-in for the library calls): once per training
loop over fixed links, again after an in-place change, after another
set_links between the forward and the backward pass, for a new tensor, and
on every forward pass with reuse_links=False."""
import pytest

torch = pytest.importorskip("torch")

from paper_1808_05506_gb300 import Dirac  # noqa: E402
from paper_1808_05506_gb300.autograd import dirac_apply  # noqa: E402


class CountingDirac(Dirac):
    """Dirac with the C calls replaced: apply multiplies by the sum of the
    loaded links, so a stale load shows in the result."""

    def __init__(self):
        self.op, self.L, self.Nv, self.Nc = "wilson", (2, 2, 2, 2), 1, 3
        self.canon_dtype = torch.complex128
        self.links_generation = 0
        self._links = None
        self.loads = 0
        self.loaded = None

    def _load_links(self, Vc, prec):
        self.loads += 1
        self.loaded = Vc.detach().clone()

    def apply(self, x, out=None, dagger=False, layout=None):
        return x * self.loaded.sum()

    def apply_dagger(self, x, out=None, layout=None):
        return x * self.loaded.sum().conj()

    def force(self, psi, g, out=None):
        return torch.zeros_like(self.loaded)

    def close(self):
        pass


def _links(seed):
    g = torch.Generator().manual_seed(seed)
    return torch.randn(2, 2, 2, 2, 4, 3, 3, dtype=torch.complex128, generator=g)


def _step(D, psi, V, **kw):
    out = dirac_apply(D, psi, V, **kw)
    out.abs().sum().backward()
    return out.detach()


def test_fixed_links_load_once():
    D = CountingDirac()
    V = _links(1).requires_grad_(True)
    psi = torch.ones(2, 2, 2, 2, 1, 4, 3, dtype=torch.complex128, requires_grad=True)
    for _ in range(3):
        out = _step(D, psi, V)
    assert D.loads == 1
    assert torch.equal(out, psi.detach() * V.detach().sum())


def test_in_place_change_reloads():
    D = CountingDirac()
    V = _links(2).requires_grad_(True)
    psi = torch.ones(2, 2, 2, 2, 1, 4, 3, dtype=torch.complex128)
    _step(D, psi, V)
    with torch.no_grad():
        V.mul_(2.0)                      # advances V's version counter
    out = _step(D, psi, V)
    assert D.loads == 2
    assert torch.equal(out, psi * V.detach().sum())


def test_other_links_between_forward_and_backward():
    D = CountingDirac()
    V = _links(3).requires_grad_(True)
    psi = torch.ones(2, 2, 2, 2, 1, 4, 3, dtype=torch.complex128, requires_grad=True)
    out = dirac_apply(D, psi, V)
    D.set_links(_links(4))               # the handle is reused before the backward pass
    out.abs().sum().backward()
    assert D.loads == 3                  # V, the other links, V again for the backward pass
    assert torch.equal(D.loaded, V.detach())


def test_new_tensor_reloads():
    D = CountingDirac()
    psi = torch.ones(2, 2, 2, 2, 1, 4, 3, dtype=torch.complex128)
    _step(D, psi, _links(5).requires_grad_(True))
    V = _links(6).requires_grad_(True)
    out = _step(D, psi, V)
    assert D.loads == 2
    assert torch.equal(out, psi * V.detach().sum())


def test_no_reuse_loads_every_time_and_is_not_remembered():
    D = CountingDirac()
    V = _links(7).requires_grad_(True)
    psi = torch.ones(2, 2, 2, 2, 1, 4, 3, dtype=torch.complex128)
    _step(D, psi, V, reuse_links=False)
    V.data.mul_(3.0)                     # not seen by the version counter
    _step(D, psi, V, reuse_links=False)
    assert D.loads == 2
    out = _step(D, psi, V)               # a reuse call after reuse_links=False loads again
    assert D.loads == 3
    assert torch.equal(out, psi * V.detach().sum())
