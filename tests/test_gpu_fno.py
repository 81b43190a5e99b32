"""GPU parity of the learned surrogate (lbm_fno_*) against the FP64 reference.

- The BF16 matrix product (lbm_fno_gemm, tcgen05 with TMA-staged operands),
  every transpose combination, FP32 and BF16 outputs, batch strides, split-K,
  ragged sizes (multiples of 16), several tiles each way, more K stages than
  the ring holds, an operand shared by the batch and one whose batch entries
  interleave along its rows, against float64 products of the same
  BF16-rounded inputs: FP32 output within 1e-5 relative (FP32
  accumulation), BF16 output within 1e-2.
- The surrogate step (lbm_fno_advance) against oracle/fno_ref.advance, the
  loss and the parameter gradient (lbm_fno_accumulate) against
  oracle/fno_ref.loss_and_grad (float64, FFT-based, autodiff pinned to finite
  differences) on a small model (32 x 48 nodes, C = 16, K = 8, L = 2: the
  separate pointwise and x-reconstruction products) and a tall one (128 x 512,
  L = 1: the two fused into one two-segment product, the y projections split
  over blocks).  The
  kernels round weights and activations to BF16 (8 significant bits), so the
  bars are relative L2 3e-2 on the state increment and the gradient of every
  parameter block, 2e-2 on the loss.
- One Adam step against the textbook update of the gradients the library
  returned; the mass-drift test of the fallback against the drift recomputed
  from the returned state.
"""
import numpy as np
import pytest
import torch

import paper_2409_10399_gb300 as lbm
from oracle import fno_ref

pytestmark = pytest.mark.gpu

DIMS = (32, 48, 16, 8, 2)  # nx, ny, C, K, L
TALL = (128, 512, 16, 8, 1)  # nx % 128 == 0: pointwise + x reconstruction fused; ny >= 512: split y projection


def _bf(t):
    return t.to(torch.bfloat16)


@pytest.mark.parametrize("ta", [False, True])
@pytest.mark.parametrize("tb", [False, True])
@pytest.mark.parametrize("out", ["f32", "bf16"])
def test_gemm_against_float64(ta, tb, out):
    g = torch.Generator(device="cpu").manual_seed(7)
    M, N, K, batch = 48, 80, 96, 3
    A = _bf(torch.randn((batch, K, M) if ta else (batch, M, K), generator=g)).cuda()
    B = _bf(torch.randn((batch, N, K) if tb else (batch, K, N), generator=g)).cuda()
    C0 = torch.randn((batch, M, N), generator=g)
    C = C0.to(torch.float32 if out == "f32" else torch.bfloat16).cuda()
    lbm.fno_gemm(A, B, C, ta=ta, tb=tb, alpha=0.5, beta=0.25, batch=batch, M=M, N=N, K=K)
    torch.cuda.synchronize()
    a = A.double().cpu()
    b = B.double().cpu()
    ref = 0.5 * torch.matmul(a.transpose(1, 2) if ta else a, b.transpose(1, 2) if tb else b) + \
        0.25 * C0.to(C.dtype).double()
    err = (C.double().cpu() - ref).norm() / ref.norm()
    assert err < (1e-5 if out == "f32" else 1e-2), err


@pytest.mark.parametrize("ta", [False, True])
@pytest.mark.parametrize("tb", [False, True])
@pytest.mark.parametrize("beta,c_side", [(0.0, False), (0.5, False), (0.5, True)])
def test_gemm_tiles_ring_and_batch_layouts(ta, tb, beta, c_side):
    """M = 192 (one full and one partial tile of output rows), N = 336 (two
    full and one partial tile of 128 columns), K = 320 (five 64-wide stages
    through a ring of four), batch 2 with A shared by the batch (stride 0)
    and B's batch entries side by side along its rows (batch stride below the
    row stride); FP32 output, with and without the old C (beta), the old C
    stacked by batch entry or side by side like B."""
    g = torch.Generator(device="cpu").manual_seed(9)
    M, N, K, batch = 192, 336, 320, 2
    A = _bf(torch.randn((K, M) if ta else (M, K), generator=g)).cuda()
    w = K if tb else N
    Bbig = _bf(torch.randn((N if tb else K, batch * w), generator=g)).cuda()
    C0 = torch.randn((batch, M, N), generator=g)
    if c_side:
        Cbig = torch.cat([C0[b] for b in range(batch)], dim=1).float().cuda()  # M x (batch N)
        lbm.fno_gemm(A, Bbig, Cbig, ta=ta, tb=tb, alpha=0.5, beta=beta, batch=batch, sB=w, sC=N, M=M, N=N, K=K)
        torch.cuda.synchronize()
        got = [Cbig[:, b * N:(b + 1) * N] for b in range(batch)]
    else:
        C = C0.float().cuda()
        lbm.fno_gemm(A, Bbig, C, ta=ta, tb=tb, alpha=0.5, beta=beta, batch=batch, sB=w, M=M, N=N, K=K)
        torch.cuda.synchronize()
        got = [C[b] for b in range(batch)]
    a = A.double().cpu()
    a = a.T if ta else a
    err = 0.0
    for b in range(batch):
        bb = Bbig[:, b * w:(b + 1) * w].double().cpu()
        ref = 0.5 * (a @ (bb.T if tb else bb)) + beta * C0[b].double()
        err = max(err, ((got[b].double().cpu() - ref).norm() / ref.norm()).item())
    assert err < 1e-5, err


def test_gemm_split_k_and_strided_rows():
    g = torch.Generator(device="cpu").manual_seed(8)
    M, N, K = 32, 64, 4096
    A = _bf(torch.randn((M, K), generator=g)).cuda()
    Bfull = _bf(torch.randn((N, K + 64), generator=g)).cuda()   # ldb > K
    C0 = torch.randn((M, N), generator=g).float().cuda()
    C = C0.clone()
    lbm.fno_gemm(A, Bfull, C, tb=True, beta=1.0, ksplit=7, M=M, N=N, K=K, ldb=K + 64)
    torch.cuda.synchronize()
    ref = A.double() @ Bfull[:, :K].double().T + C0.double()
    assert ((C.double() - ref).norm() / ref.norm()).item() < 1e-5
    with pytest.raises(lbm.LBMError):
        lbm.fno_gemm(A, Bfull, C, tb=True, beta=0.0, ksplit=7, M=M, N=N, K=K, ldb=K + 64)  # split needs beta = 1
    with pytest.raises(lbm.LBMError):
        lbm.fno_gemm(A, Bfull, C, tb=True, M=M, N=N, K=40, ldb=K + 64)                     # K not a multiple of 16


def _case(seed=11, scale=0.5, dims=DIMS):
    nx, ny, C, K, L = dims
    r = np.random.default_rng(seed)
    n = sum(int(np.prod(s)) for _, s in fno_ref.layout(C, K, L))
    p = (r.standard_normal(n) * scale / np.sqrt(C)).astype(np.float32)
    P = nx * ny
    x = (np.arange(P) % nx) / nx
    y = (np.arange(P) // nx) / ny
    norm = (np.array([0.3, 0, 0, 0, 0, 1 / 3]), np.array([0.1, 1e-3, 1e-3, 5e-4, 5e-4, 1e-6]),
            np.array([1e-3, 1e-4, 1e-4, 5e-5, 5e-5, 1e-7]))
    now = np.stack([0.3 + 0.1 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y),
                    1e-3 * np.sin(2 * np.pi * y), 1e-3 * np.cos(2 * np.pi * x),
                    -5e-4 * np.sin(2 * np.pi * y), 2e-4 * np.cos(2 * np.pi * x),
                    1 / 3 + 1e-6 * np.sin(2 * np.pi * (x + y))])
    now = now + 0.1 * norm[1][:, None] * r.standard_normal((6, P))
    nxt = now + norm[2][:, None] * r.standard_normal((6, P))
    return p, now, nxt, norm


def _model(p, norm, dims=DIMS):
    nx, ny, C, K, L = dims
    m = lbm.Surrogate(nx, ny, C, K, L)
    m.set_params(p)
    m.set_norm(*norm)
    return m


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dims", [DIMS, TALL])
def test_advance_against_reference(dims):
    p, now, _, norm = _case(dims=dims)
    m = _model(p, norm, dims)
    now_d = torch.from_numpy(now).cuda().contiguous()
    out = torch.empty_like(now_d)
    drift, ok = m.advance(now_d, out, max_drift=1.0)
    got = out.cpu().numpy()
    ref = fno_ref.advance(p.astype(np.float64), now, dims, norm)
    for c in range(6):
        assert _rel(got[c] - now[c], ref[c] - now[c]) < 3e-2, c
    s0, s1 = now[0].sum(), got[0].sum()
    expect = max(abs(s1 - s0) / s0, abs(s1 - s0) / (now.shape[1] - s0))
    assert abs(drift - expect) <= 1e-9 * max(expect, 1e-30) + 1e-15
    assert ok == (expect <= 1.0)
    _, ok0 = m.advance(now_d, out, max_drift=0.0)
    assert not ok0  # any change of sum(alpha_g) fails a zero tolerance
    # an expected inflow: the check tests the change beyond it
    for dV in (s1 - s0, 0.5 * (s1 - s0) + 1.0):
        m.set_inflow(dV)
        d_in, _ = m.advance(now_d, out, max_drift=1.0)
        ex = abs((s1 - s0) - dV)
        assert abs(d_in - max(ex / s0, ex / (now.shape[1] - s0))) <= 1e-9 * max(ex / s0, 1e-30) + 1e-13
    m.set_inflow(0.0)
    bad = now_d.clone()
    bad[3, 5] = float("nan")  # a liquid velocity, not alpha_g
    d_bad, ok_bad = m.advance(bad, out, max_drift=1e30)
    assert not ok_bad and d_bad == float("inf")


# cons = 5: the conservation term's gradient (a uniform 2 cons mean(e_0) / P on
# the alpha_g channel) then outweighs the squared error's on that channel,
# while the input blocks whose BF16-rounded inputs sum to nearly zero over the
# nodes (W_in's p_k column) stay inside the bar; at cons = 50 that column's
# cancellation against BF16 rounding reached 3.6 %.
@pytest.mark.parametrize("dims,cons", [(DIMS, 0.0), (TALL, 0.0), (DIMS, 5.0)])
def test_loss_and_gradient_against_reference(dims, cons):
    p, now, nxt, norm = _case(seed=12, dims=dims)
    m = _model(p, norm, dims)
    m.set_loss(cons)
    m.zero_grads()
    loss = m.accumulate(torch.from_numpy(now).cuda().contiguous(), torch.from_numpy(nxt).cuda().contiguous())
    g = m.grads()
    ref_loss, ref_g = fno_ref.loss_and_grad(p.astype(np.float64), now, nxt, dims, norm, cons)
    assert abs(loss - ref_loss) <= 2e-2 * ref_loss, (loss, ref_loss)
    nx, ny, C, K, L = dims
    at = 0
    for name, shape in fno_ref.layout(C, K, L):
        n = int(np.prod(shape))
        a, b = g[at:at + n], ref_g[at:at + n]
        at += n
        if np.linalg.norm(b) == 0.0:
            continue
        if name.startswith("B") and name[1] in "xy":
            # mode 0 of B_k has no effect (sin 0 = 0): its gradient is zero on both sides
            b0, a0 = b.reshape(shape)[0], a.reshape(shape)[0]
            assert np.abs(a0).max() <= 1e-6 * np.abs(b).max() + 1e-30 and np.abs(b0).max() < 1e-9 * np.abs(b).max()
        assert _rel(a, b) < 3e-2, (name, _rel(a, b))


def test_adam_step_is_the_textbook_update():
    p, now, nxt, norm = _case(seed=13)
    m = _model(p, norm)
    m.zero_grads()
    m.accumulate(torch.from_numpy(now).cuda().contiguous(), torch.from_numpy(nxt).cuda().contiguous())
    g = m.grads().astype(np.float64) * 0.5
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    m.adam(lr, b1, b2, eps, grad_scale=0.5)
    mt, vt = (1 - b1) * g, (1 - b2) * g * g
    ref = p - lr * np.sqrt(1 - b2) / (1 - b1) * mt / (np.sqrt(vt) + eps)
    got = m.params()
    assert np.allclose(got, ref, rtol=1e-5, atol=1e-7)
    assert np.abs(m.grads()).max() == 0.0  # zeroed after the step


def _lattice(dims=DIMS, seed=5, prec="fp64", **extra):
    import lbm_inputs
    from paper_2409_10399_gb300 import surrogate as S
    nx, ny = dims[0], dims[1]
    sim = lbm.Simulation("D2Q9", (nx, ny), dict(S._lbm_params(prec, recipe="plume"), **extra))
    sim.init(**lbm_inputs.fields_plumes(nx, ny, seed))
    return sim


def _state_of(sim):
    m = sim.moments()
    return np.concatenate([m["alpha_g"][None], m["u_g"], m["u_l"], m["p_k"][None]])


def test_surrogate_window_on_a_lattice_takes_the_model_state():
    p, _, _, norm = _case(seed=14)
    m = _model(p, norm)
    sim = _lattice()
    now = _state_of(sim)
    drift, used = m.advance_lattice(sim, 64, max_drift=1e30)
    assert used and sim.t == 64
    # the same fields through lbm_init on a twin lattice: identical moments
    pred = torch.empty((6, now.shape[1]), dtype=torch.float64, device="cuda")
    d2, _ = m.advance(torch.from_numpy(now).cuda().contiguous(), pred, max_drift=1e30)
    assert d2 == drift
    pred = pred.cpu().numpy()
    twin = _lattice()
    twin.init(alpha_g=pred[0], u_g=pred[1:3], u_l=pred[3:5], p_k=pred[5])
    assert np.array_equal(_state_of(sim), _state_of(twin))


def test_surrogate_window_on_an_fp32_lattice():
    # the workload's store: deviations from a reference set to the predicted
    # mean alpha_g, summed on the device by the window and on the host by
    # lbm_init, so the twin agrees to FP32 rounding rather than bit for bit
    p, _, _, norm = _case(seed=17)
    m = _model(p, norm)
    sim = _lattice(prec="fp32")
    now = _state_of(sim)
    _, used = m.advance_lattice(sim, 64, max_drift=1e30)
    assert used and sim.t == 64
    pred = torch.empty((6, now.shape[1]), dtype=torch.float64, device="cuda")
    m.advance(torch.from_numpy(now).cuda().contiguous(), pred, max_drift=1e30)
    pred = pred.cpu().numpy()
    twin = _lattice(prec="fp32")
    twin.init(alpha_g=pred[0], u_g=pred[1:3], u_l=pred[3:5], p_k=pred[5])
    a, b = _state_of(sim), _state_of(twin)
    assert np.abs(a[0] - b[0]).max() <= 1e-6 * np.abs(b[0]).max()
    assert _rel(a[1:5], b[1:5]) < 1e-5
    sim.step(64)  # the lattice carries on from the re-initialised state
    assert np.isfinite(_state_of(sim)).all() and sim.t == 128


@pytest.mark.parametrize("prec,bstencil", [("fp64", 0), ("fp64dev", 0), ("fp64dev", 1)])
def test_surrogate_reinit_steps_like_a_fresh_init(prec, bstencil):
    """After an accepted window the lattice is re-initialised at clock
    t + window (64 here, not a multiple of n_gamma = 200).  Its next steps must
    be those of a twin given the same fields by lbm_init at t = 0: the first
    step after either initialisation latches S'' and Lambda' (Eq.
    (lbm-cont-1D-update)) and, in the beta-stencil form, evaluates the
    streamed beta populations from each node's own c (the initial state holds
    f^eq(1, c(x)) at x).  Twenty steps stay before the next latch of either
    clock.  FP64: bitwise.  FP64-deviation forms: the deviation reference is
    the predicted mean alpha_g, summed on the device by the window and on the
    host by lbm_init, so the two agree to double rounding (1e-12)."""
    p, _, _, norm = _case(seed=18)
    m = _model(p, norm)
    sim = _lattice(prec=prec, beta_stencil=bstencil)
    now = _state_of(sim)
    _, used = m.advance_lattice(sim, 64, max_drift=1e30)
    assert used and sim.t == 64
    pred = torch.empty((6, now.shape[1]), dtype=torch.float64, device="cuda")
    m.advance(torch.from_numpy(now).cuda().contiguous(), pred, max_drift=1e30)
    pred = pred.cpu().numpy()
    twin = _lattice(prec=prec, beta_stencil=bstencil)
    twin.init(alpha_g=pred[0], u_g=pred[1:3], u_l=pred[3:5], p_k=pred[5])
    sim.step(20)
    twin.step(20)
    assert sim.t == 84 and twin.t == 20
    a, b = sim.moments(), twin.moments()
    for k in ("alpha_g", "u_g", "u_l", "p_k", "S_g", "S_l"):
        if prec == "fp64":
            assert np.array_equal(a[k], b[k]), k
        else:
            ref = b[k] - (1 / 3 if k == "p_k" else 0.0)
            assert np.linalg.norm(a[k] - b[k]) <= 1e-12 * np.linalg.norm(ref), k


def test_surrogate_window_falls_back_to_the_lattice_steps():
    p, _, _, norm = _case(seed=15)
    m = _model(p, norm)
    sim, twin = _lattice(), _lattice()
    drift, used = m.advance_lattice(sim, 64, max_drift=0.0)  # any volume change fails
    assert not used and drift > 0.0 and sim.t == 64
    twin.step(64)
    assert np.array_equal(_state_of(sim), _state_of(twin))  # the LBM from its own populations


def test_surrogate_window_rejects_other_lattices_and_odd_times():
    p, _, _, norm = _case(seed=16)
    m = _model(p, norm)
    sim = _lattice()
    sim.step(1)
    with pytest.raises(lbm.LBMError) as e:
        m.advance_lattice(sim, 64)
    assert e.value.code == -7  # LBM_ESTATE: populations mid-swap at odd t
    with pytest.raises(lbm.LBMError) as e:
        m.advance_lattice(_lattice((48, 32)), 64)
    assert e.value.code == -1  # LBM_EINVAL: not the model's grid
    with pytest.raises(lbm.LBMError) as e:
        m.advance_lattice(_lattice(), 63)
    assert e.value.code == -1
