"""Time-dependent Hamiltonian inside a captured CUDA graph (Sec. I: time-dependent Hamiltonians): a
Peierls-phased pulse on the boundary hopping, a(t) = t exp(i A sin(w t)) and its Hermitian partner
-conj(a(t)), with the connection coefficients read at run time from a device array
(tdmrg_set_coefficients).  One graph holds a whole time step: copy step k's coefficients from a device
schedule into the registered array, advance the step counter, Krylov advance.  Eight replays against
the oracle evolving with the same coefficients.  Bounds: FP64 path 1e-10 relative per target; tensor
path (4 slices) 1.1e-6, as in the bench-trajectory test.  Also: registering an array equal to the
static coefficients changes no bit of H psi on the FP64 path, and stays within the slicing bound
(140 2^-28) on the tensor path, which then slices the coefficients with the intermediates."""
import numpy as np
import pytest

from oracle import krylov, superblock
from tests.gpu_util import dev, host, new_ctx, oracle_ops_of_synthetic, rel_err, torch_cuda
from workloads import sectors as S

pytestmark = pytest.mark.gpu
STEPS, TAU = 8, 0.05


@pytest.fixture(scope="module")
def lib():
    from paper_1103_5391_gb300 import tdmrg as T
    return T


def _pulse(t0, k):
    a = t0 * np.exp(1j * 0.8 * np.sin(3.0 * k * TAU))
    return a


@pytest.mark.parametrize("slices", [0, 4])
def test_static_equal_device_coefficients(lib, slices):
    torch = torch_cuda()
    from paper_1103_5391_gb300 import problem
    ss = S.make_synthetic(16, 120, 4.0, nbonds=1, seed=S.SEED_BASE + 8)
    kw = dict(prec=lib.TDMRG_OZAKI_BF16, ozaki_slices=slices) if slices else {}
    ctx = new_ctx(**kw)
    try:
        gconns = problem.load_synthetic(ctx, ss)
        n = lib.tdmrg_sector_size(ctx, ss.Q1)
        x = dev(ss.phi)
        y0, y1 = dev(np.zeros(n)), dev(np.zeros(n))
        lib.tdmrg_apply_h(ctx, ss.Q1, x, y0)
        coef = torch.tensor([complex(c) for _, _, c in gconns], dtype=torch.complex128, device="cuda")
        lib.tdmrg_set_coefficients(ctx, coef)
        lib.tdmrg_apply_h(ctx, ss.Q1, x, y1)
        if slices == 0:
            assert np.array_equal(host(y0).view(np.float64), host(y1).view(np.float64))
        else:
            assert rel_err(host(y1), host(y0)) < 140.0 * 2.0 ** -28
    finally:
        lib.tdmrg_destroy(ctx)


@pytest.mark.parametrize("slices", [0, 4])
def test_pulse_in_captured_graph(lib, slices):
    torch = torch_cuda()
    from paper_1103_5391_gb300 import problem
    ss = S.make_synthetic(16, 120, 4.0, nbonds=1, seed=S.SEED_BASE + 8)
    sb, HL, HR, conns = oracle_ops_of_synthetic(ss)
    times = krylov.target_times(TAU, 4)
    # oracle: step k evolves under the pulse value of step k
    refs, cur = [], ss.phi
    for k in range(STEPS):
        a = _pulse(ss.coeff_t, k)
        ck = [((a if i % 2 == 0 else -np.conj(a)), A, B) for i, (_, A, B) in enumerate(conns)]
        tg, _, _ = krylov.evolve(lambda v: superblock.apply_h(sb, HL, HR, ck, ss.Q1, v), cur, times, 10)
        refs.append(tg)
        cur = tg[-1]
    kw = dict(prec=lib.TDMRG_OZAKI_BF16, ozaki_slices=slices) if slices else {}
    ctx = new_ctx(**kw)
    stream = torch.cuda.current_stream()
    try:
        gconns = problem.load_synthetic(ctx, ss)
        nconn = len(gconns)
        sched = torch.tensor([[(_pulse(ss.coeff_t, k) if i % 2 == 0 else -np.conj(_pulse(ss.coeff_t, k)))
                               for i in range(nconn)] for k in range(STEPS)], dtype=torch.complex128, device="cuda")
        coef = sched[0].clone()
        step = torch.zeros(1, dtype=torch.int64, device="cuda")
        lib.tdmrg_set_coefficients(ctx, coef)
        n = lib.tdmrg_sector_size(ctx, ss.Q1)
        phi = dev(ss.phi)
        tg = [dev(np.zeros(n)) for _ in range(3)] + [phi]
        # one direct step builds the plans and workspace; then restart from phi0
        lib.tdmrg_evolve(ctx, ss.Q1, phi, times, 10, tg)
        torch.cuda.synchronize()
        phi.copy_(dev(ss.phi))
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        lib.tdmrg_set_stream(ctx, side.cuda_stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side, capture_error_mode="thread_local"):
            coef.copy_(torch.index_select(sched, 0, step).view(-1))
            step.add_(1)
            lib.tdmrg_evolve(ctx, ss.Q1, phi, times, 10, tg)
        lib.tdmrg_set_stream(ctx, stream.cuda_stream)
        torch.cuda.synchronize()
        bound = 1e-10 if not slices else 1.1e-6
        for k in range(STEPS):
            graph.replay()
            torch.cuda.synchronize()
            for x in range(4):
                assert rel_err(host(tg[x]), refs[k][x]) < bound, (k, x)
        assert step.item() == STEPS
        lib.tdmrg_evolve_info(ctx)
        # the pulse mattered: the last state differs from evolving with the static coefficients
        cur = ss.phi
        for k in range(STEPS):
            cur = krylov.evolve(lambda v: superblock.apply_h(sb, HL, HR, conns, ss.Q1, v), cur, times, 10)[0][-1]
        assert rel_err(refs[-1][-1], cur) > 1e-3
    finally:
        lib.tdmrg_destroy(ctx)
