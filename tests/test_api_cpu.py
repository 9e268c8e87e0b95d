"""The autograd wrappers' plumbing on CPU with a stand-in pipeline (no library calls): the
geometry-differentiable solve passes the seven differentiable inputs to the scene build and
hands each gradient of rgs_adjoint_geometry back to its input."""
import pytest

torch = pytest.importorskip("torch")

from paper_2509_18497_gb300 import api  # noqa: E402


class FakePipeline:
    built = None

    def __init__(self, alpha_model, pairs=False):
        self.alpha_model, self.pairs = alpha_model, pairs

    def build(self, d):
        FakePipeline.built = d

    def trace(self, d):
        pass

    def solve(self, E, nb):
        n = FakePipeline.built["p"].shape[0]
        return torch.full((n, 4, 3), 1.0), None

    def adjoint_geometry(self, g):
        n = g.shape[0]
        mk = lambda *shape, v: torch.full(shape, float(v))  # noqa: E731
        return (mk(n, 4, 3, v=1), mk(n, 3, v=2), mk(n, v=3), mk(n, 3, v=4), mk(n, 2, v=5), mk(n, 3, v=6),
                mk(n, 3, v=7))


def test_geometry_autograd_plumbing(monkeypatch):
    monkeypatch.setattr(api, "Pipeline", FakePipeline)
    n = 5
    leaves = dict(E=torch.zeros(n, 4, 3), ad=torch.zeros(n, 3), o=torch.zeros(n), p=torch.arange(15.0).reshape(n, 3),
                  s=torch.ones(n, 2), tu=torch.eye(3)[[0] * n], tv=torch.eye(3)[[1] * n])
    for v in leaves.values():
        v.requires_grad_(True)
    geom = dict(p=None, s=None, tu=None, tv=None, ad=None, o=None, k=torch.ones(n), light_pos=torch.zeros(1, 3))
    B = api.radiosity_geometry(leaves["E"], leaves["ad"], leaves["o"], leaves["p"], leaves["s"], leaves["tu"],
                               leaves["tv"], geom, 2)
    assert torch.equal(FakePipeline.built["p"], leaves["p"].detach())  # the inputs reach the build
    assert not FakePipeline.built["p"].requires_grad
    assert FakePipeline.built["k"] is geom["k"]
    B.sum().backward()
    for key, v in zip(("E", "ad", "o", "p", "s", "tu", "tv"), range(1, 8)):
        assert torch.all(leaves[key].grad == v), key
