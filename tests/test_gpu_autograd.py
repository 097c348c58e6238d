"""The PyTorch autograd wrapper of the checkpointed objective: its value and gradients equal the C-ABI
objective and adjoint, and torch.autograd.gradcheck (central differences of the FP64 forward) agrees
with the adjoint gradient for the porosity and the inlet velocity. The inputs are CUDA tensors and
the gradients come back on the device (the wrapper hands pointers to the library; no host copies)."""
import numpy as np
import pytest

from paper_2506_21804_gb300 import inputs as I

pytestmark = pytest.mark.gpu

lbm = pytest.importorskip("paper_2506_21804_gb300.lbm")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    lbm.lib()


def _duct():
    d = I.duct(n=6, u_in=0.03, tau=0.7, sigma=1.5, cs=0.1, dtype=np.float64)
    lat = lbm.Lattice.from_workload(d, storage=lbm.F64)
    return d, lat


def test_autograd_matches_c_abi_objective_and_adjoint():
    from paper_2506_21804_gb300.autograd import pressure_drop
    d, lat = _duct()
    T, W, xa, xb = 12, 4, 1, d.nx - 2
    gamma = torch.tensor(np.asarray(d.gamma), dtype=torch.float64, device="cuda", requires_grad=True)
    u_in = torch.tensor(np.asarray(d.uin), dtype=torch.float64, device="cuda", requires_grad=True)
    J = pressure_drop(gamma, u_in, lat, d.rho0, d.u0, T, W, xa, xb, 2)
    assert J.device.type == "cuda"
    J.backward()
    assert gamma.grad.device.type == "cuda" and u_in.grad.device.type == "cuda"
    ref = lbm.Lattice.from_workload(d, storage=lbm.F64)
    Jr = ref.objective_forward(T, W, xa, xb, ckpt=2)
    gr, ur = ref.objective_backward()
    assert abs(J.item() - Jr) < 1e-15 * max(1.0, abs(Jr))
    assert np.abs(gamma.grad.cpu().numpy() - gr).max() < 1e-14
    assert np.abs(u_in.grad.cpu().numpy() - ur).max() < 1e-14


def test_autograd_fp32_lattice_device_tensors():
    """FP32 lattice with FP32 CUDA inputs: gradients are FP32 CUDA tensors equal (to FP32 rounding of
    the FP64 accumulators) to the C ABI's FP64 gradients of the same run."""
    from paper_2506_21804_gb300.autograd import pressure_drop
    d = I.duct(n=8, u_in=0.03, tau=0.7, sigma=1.5, cs=0.1, dtype=np.float32)
    lat = lbm.Lattice.from_workload(d, storage=lbm.F32)
    T, W, xa, xb = 16, 4, 1, d.nx - 2
    gamma = torch.tensor(np.asarray(d.gamma, np.float32), device="cuda", requires_grad=True)
    u_in = torch.tensor(np.asarray(d.uin, np.float32), device="cuda", requires_grad=True)
    J = pressure_drop(gamma, u_in, lat, np.asarray(d.rho0, np.float32), np.asarray(d.u0, np.float32), T, W, xa, xb, 2)
    J.backward()
    assert gamma.grad.device.type == "cuda" and gamma.grad.dtype == torch.float32
    ref = lbm.Lattice.from_workload(d, storage=lbm.F32)
    ref.set_porosity(np.asarray(d.gamma, np.float32))
    Jr = ref.objective_forward(T, W, xa, xb, ckpt=2)
    gr, ur = ref.objective_backward()
    assert abs(J.item() - Jr) <= 1e-6 * max(1.0, abs(Jr))
    assert np.abs(gamma.grad.cpu().numpy() - gr).max() <= 1e-6 * np.abs(gr).max()
    assert np.abs(u_in.grad.cpu().numpy() - ur).max() <= 1e-6 * np.abs(ur).max()


def test_autograd_gradcheck_fp64():
    from paper_2506_21804_gb300.autograd import pressure_drop
    d, lat = _duct()
    T, W, xa, xb = 8, 4, 1, d.nx - 2
    gamma = torch.tensor(np.asarray(d.gamma), dtype=torch.float64, device="cuda", requires_grad=True)
    u_in = torch.tensor(np.asarray(d.uin), dtype=torch.float64, device="cuda", requires_grad=True)
    fn = lambda g, u: pressure_drop(g, u, lat, d.rho0, d.u0, T, W, xa, xb, 2)  # noqa: E731
    assert torch.autograd.gradcheck(fn, (gamma, u_in), eps=1e-6, atol=1e-9, rtol=1e-3)
