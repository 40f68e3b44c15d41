"""The allocation-free Jacobian entry point agrees with the context-based one (GPU).

dino_surrogate_jacobian_noalloc serves callers that must not allocate device
memory (a plugin whose host framework owns all device memory, a loop that
cannot afford cudaMalloc's synchronisation).  It keeps its intermediates in a
fixed device array; this test feeds it caller-owned device buffers (allocated
here by torch, which the entry point itself never calls) and compares f and J
with dino_surrogate_eval on the same surrogate, within the FP64 parity bar,
on two calls in a row.  The file is named to run last.
"""
import numpy as np
import pytest

from helpers import rel_err
from workloads import BASIS_KLE, CONFIGS, surrogate_inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def test_noalloc_matches_context_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    import paper_2403_08220_gb300 as dino

    w = CONFIGS["r200_kle_fp64"]            # GELU 200-400-400-100
    inp = surrogate_inputs(w)
    ctx = dino.dino_init(0)
    try:
        sid = dino.dino_load_surrogate(
            ctx, n_grid=w.n_grid, prior_gamma=w.prior_gamma, prior_delta=w.prior_delta,
            r=w.r, widths=w.widths, activation=w.activation, W=inp["Ws"], b=inp["bs"],
            basis_kind=BASIS_KLE, precision=dino.DINO_PREC_FP64)
        dev = torch.device("cuda", 0)
        Wt = [torch.tensor(W, dtype=torch.float64, device=dev).contiguous() for W in inp["Ws"]]
        bt = [torch.tensor(b, dtype=torch.float64, device=dev).contiguous() for b in inp["bs"]]
        n = 8                                   # 8 * 2 * 100 * 400 doubles fit the 8 MiB scratch
        rng = np.random.default_rng(42)
        for call in range(2):
            x = rng.standard_normal((n, w.r))
            ref = dino.dino_surrogate_eval(ctx, sid, x, w.d_y, want_L=False)
            xt = torch.tensor(x, dtype=torch.float64, device=dev)
            ft = torch.full((n, w.d_y), float("nan"), dtype=torch.float64, device=dev)
            Jt = torch.full((n, w.d_y, w.r), float("nan"), dtype=torch.float64, device=dev)
            stream = torch.cuda.current_stream().cuda_stream
            dino.dino_surrogate_jacobian_noalloc(
                n, w.widths, w.activation, [t.data_ptr() for t in Wt],
                [t.data_ptr() for t in bt], xt.data_ptr(), ft.data_ptr(), Jt.data_ptr(), stream)
            torch.cuda.synchronize()
            assert rel_err(ft.cpu().numpy(), ref["f"]) <= TOL, f"f differs on call {call}"
            assert rel_err(Jt.cpu().numpy(), ref["J"]) <= TOL, f"J differs on call {call}"
        # a request beyond the fixed scratch is refused before anything runs
        big = 64
        xt = torch.zeros((big, w.r), dtype=torch.float64, device=dev)
        ft = torch.zeros((big, w.d_y), dtype=torch.float64, device=dev)
        Jt = torch.zeros((big, w.d_y, w.r), dtype=torch.float64, device=dev)
        with pytest.raises(dino.DinoError) as e:
            dino.dino_surrogate_jacobian_noalloc(
                big, w.widths, w.activation, [t.data_ptr() for t in Wt],
                [t.data_ptr() for t in bt], xt.data_ptr(), ft.data_ptr(), Jt.data_ptr(), 0)
        assert e.value.code == dino.DINO_ENOMEM
    finally:
        ctx.close()
