"""The allocation-free Jacobian entry point against the FP64 oracle (GPU).

dino_surrogate_jacobian_noalloc serves callers that must not allocate device
memory (a plugin whose host framework owns all device memory, a loop that
cannot afford cudaMalloc's synchronisation).  It keeps its intermediates in a
fixed device array.  This test feeds it caller-owned device buffers
(allocated here by torch, which the entry point itself never calls) and
compares f and J with the oracle's forward pass and reverse-mode Jacobian
within the FP64 parity bar, on two calls in a row, for each activation, a
single affine layer, and a hidden layer wide enough that the activations
need more than 48 KB of shared memory.  It also checks, on the GELU network,
that the context-based entry point gives the same values.  The file is named
to run last.
"""
import numpy as np
import pytest

from helpers import rel_err
from oracle import mlp
from workloads import BASIS_KLE, CONFIGS, mlp_weights, surrogate_inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10

# (widths, activation, points per call); scratch use n * 2 * d_y * widest hidden
# must stay within 2^20 doubles
CASES = {
    "gelu_200_400_400_100": ([200, 400, 400, 100], mlp.ACT_GELU, 8),
    "tanh_16_64_64_49": ([16, 64, 64, 49], mlp.ACT_TANH, 16),
    "identity_12_30_7": ([12, 30, 7], mlp.ACT_IDENTITY, 5),
    "one_layer_20_9": ([20, 9], mlp.ACT_TANH, 3),
    "wide_64_3200_4": ([64, 3200, 4], mlp.ACT_GELU, 6),   # 51.7 KB of activations
}


def _oracle(Ws, bs, act, x):
    f, zs = mlp.forward(Ws, bs, act, x)
    if len(Ws) == 1:
        J = np.broadcast_to(Ws[0], (x.shape[0],) + Ws[0].shape)
    else:
        J = mlp.jacobian_reverse(Ws, act, zs)
    return f, J


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_matches_oracle_on_two_calls(name):
    torch = pytest.importorskip("torch")
    import paper_2403_08220_gb300 as dino

    widths, act, n = CASES[name]
    Ws, bs = mlp_weights(widths, 40 + len(name))
    r, dy = widths[0], widths[-1]
    dev = torch.device("cuda", 0)
    Wt = [torch.tensor(W, dtype=torch.float64, device=dev).contiguous() for W in Ws]
    bt = [torch.tensor(b, dtype=torch.float64, device=dev).contiguous() for b in bs]
    rng = np.random.default_rng(42)
    for call in range(2):
        x = rng.standard_normal((n, r))
        f_ref, J_ref = _oracle(Ws, bs, act, x)
        xt = torch.tensor(x, dtype=torch.float64, device=dev)
        ft = torch.full((n, dy), float("nan"), dtype=torch.float64, device=dev)
        Jt = torch.full((n, dy, r), float("nan"), dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream().cuda_stream
        dino.dino_surrogate_jacobian_noalloc(
            n, widths, act, [t.data_ptr() for t in Wt], [t.data_ptr() for t in bt],
            xt.data_ptr(), ft.data_ptr(), Jt.data_ptr(), stream)
        torch.cuda.synchronize()
        assert rel_err(ft.cpu().numpy(), f_ref) <= TOL, f"f differs on call {call}"
        assert rel_err(Jt.cpu().numpy(), J_ref) <= TOL, f"J differs on call {call}"


def test_noalloc_agrees_with_context_entry_point_and_refuses_oversize():
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
        n = 8
        x = np.random.default_rng(43).standard_normal((n, w.r))
        ref = dino.dino_surrogate_eval(ctx, sid, x, w.d_y, want_L=False)
        xt = torch.tensor(x, dtype=torch.float64, device=dev)
        ft = torch.zeros((n, w.d_y), dtype=torch.float64, device=dev)
        Jt = torch.zeros((n, w.d_y, w.r), dtype=torch.float64, device=dev)
        dino.dino_surrogate_jacobian_noalloc(
            n, w.widths, w.activation, [t.data_ptr() for t in Wt], [t.data_ptr() for t in bt],
            xt.data_ptr(), ft.data_ptr(), Jt.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert rel_err(ft.cpu().numpy(), ref["f"]) <= TOL
        assert rel_err(Jt.cpu().numpy(), ref["J"]) <= TOL
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
