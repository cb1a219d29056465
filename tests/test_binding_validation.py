"""Host-side argument checks of the Python binding (no GPU: every case is rejected before a
pointer reaches the library)."""
import pytest
import torch

from paper_2412_08264_gb300 import api


class FakeCuda:
    """Stands in for a CUDA tensor in the binding's checks (this host has no GPU)."""

    def __init__(self, n, dtype=torch.float32, device="cuda:0", contiguous=True):
        self.n, self.dtype, self.device, self.contig = n, dtype, torch.device(device), contiguous
        self.is_cuda = True

    def numel(self):
        return self.n

    def is_contiguous(self):
        return self.contig


def bare_problem(sizes=((4, 5), (3, 3)), dtype=torch.float32, device="cuda:0", p=7):
    P = api.Problem.__new__(api.Problem)
    P.K, P.sizes, P.dtype, P.device, P.p = len(sizes), list(sizes), dtype, torch.device(device), p
    return P


@pytest.mark.parametrize("kw,msg", [(dict(reg="tikhonov"), "regulariser"), (dict(precision="fp16"), "precision"),
                                    (dict(phi="huber"), "phi")])
def test_create_rejects_unknown_options(kw, msg):
    args = dict(reg="foe", n_filters=2, filter_size=3, precision="fp32", phi="charbonnier")
    args.update(kw)
    with pytest.raises(ValueError, match=msg):
        api.Problem([(4, 4, 1.0, 1)], y=torch.zeros(16), x_star=torch.zeros(16), **args)


def test_image_checks():
    P = bare_problem()
    P._check_images(FakeCuda(29))
    with pytest.raises(ValueError, match="lives on"):
        P._check_images(FakeCuda(29, device="cuda:1"))
    with pytest.raises(ValueError, match="contiguous"):
        P._check_images(FakeCuda(29, contiguous=False))
    with pytest.raises(ValueError, match="expected"):
        P._check_images(FakeCuda(29, dtype=torch.float64))
    with pytest.raises(ValueError, match="elements"):
        P._check_images(FakeCuda(28))
    P._check_images(FakeCuda(9), pairs=[1])
    with pytest.raises(ValueError, match="contiguous CUDA"):
        P._check_images(torch.zeros(29))


def test_theta_checks():
    P = bare_problem()
    P._check_theta(FakeCuda(7, dtype=torch.float64))
    with pytest.raises(ValueError, match="lives on"):
        P._check_theta(FakeCuda(7, dtype=torch.float64, device="cuda:2"))
    with pytest.raises(ValueError, match="float64"):
        P._check_theta(FakeCuda(7, dtype=torch.float32))
    with pytest.raises(ValueError, match="float64"):
        P._check_theta(FakeCuda(6, dtype=torch.float64))


def test_hessian_solve_checks_nsc_scale_length():
    P = bare_problem()
    w = FakeCuda(29)
    with pytest.raises(ValueError, match="nsc_scale"):
        P.hessian_solve(w, nsc_scale=[1.0])
    with pytest.raises(ValueError, match="Krylov method"):
        P.hessian_solve(w, method="gmres")
