"""GPU checks of the learned exit proposal: first-passage data bit-exact against
the oracle, the tensor-core network's loss and gradients against the FP64
reference network, and training that learns the first-passage distribution."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import coracle as C  # noqa: E402
from oracle import mlp as M  # noqa: E402
from paper_1709_10187_gb300 import build as B  # noqa: E402
from paper_1709_10187_gb300 import learned as Lr  # noqa: E402
from paper_1709_10187_gb300 import rddmc as R  # noqa: E402
from paper_1709_10187_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

# a small clumpy-medium target: 32^3 cells, 64 bins over [-64, 64], tau0 = 1e6
TARGET = W.Workload("clumpy_small", 3, (32, 32, 32), 64, -64.0, 64.0, 1.0e6, 1.0e4, 1, 1)
RHO = np.logspace(-1.5, 1.5, 8)


@pytest.fixture(scope="module")
def proposal():
    B.build()
    return Lr.ExitProposal(TARGET, 4, RHO, tau_lo=5.0, tau_hi=120.0)


def test_first_passages_match_oracle_bit_exactly(proposal):
    p = proposal
    rows = []
    for pb, rho in zip(p.problems, p.levels):
        rows.append(C.interior_rows(pb.w))
        thr, _ = pb.rows()
        assert np.array_equal(thr.reshape(27, p.J, 7)[13], rows[-1][:, :7])
    rows = np.stack(rows)
    n = 3000
    d = p.generate(n, seed=77, p0=1000)
    out, steps = C.fp_samples(rows, p.b, p.jlo, p.jhi, 77, 1000, n, 10_000_000)
    assert np.array_equal(d["rec"].cpu().numpy(), out)
    assert np.array_equal(d["steps"].cpu().numpy().astype(np.uint64), steps)
    tA, tC = d["tA"].cpu().numpy(), d["tC"].cpu().numpy()
    ok = out[:, 3] < 6
    assert np.array_equal(tA[ok], out[ok, 3] * p.J + out[ok, 4]) and np.all(tA[~ok] == -1)
    assert np.array_equal(tC[ok], out[ok, 3] * p.S + out[ok, 5]) and np.all(tC[~ok] == -1)


def test_network_loss_and_gradients_match_fp64_reference(proposal):
    p = proposal
    rng = np.random.default_rng(5)
    Bsz = 256
    d = p.generate(Bsz, seed=91)
    X = d["X"]
    tA, tB, tC = d["tA"], d["tB"], d["tC"]
    assert p.nC == 6 * p.b * p.b
    loss = p.loss_grad(X, tA, tB, tC)
    torch.cuda.synchronize()
    g_gpu = p.grad.cpu().numpy().astype(np.float64)
    w_bf = p.wb.float().cpu().numpy().astype(np.float64)   # the weights the tensor cores saw
    w_f = p.wf.cpu().numpy().astype(np.float64)
    # biases are applied in FP32 from the master copy
    flat = w_bf.copy()
    offs, off = [], 0
    for (o, i) in M.shapes(p.n_out):
        offs.append((off + o * i, o))
        off += o * i + o
    for s, o in offs:
        flat[s:s + o] = w_f[s:s + o]
    lo, g_ref = M.loss_and_grad(flat, p.n_out, p.nA, p.nB, X.float().cpu().numpy(), tA.cpu().numpy(),
                                tB.cpu().numpy(), p.nC, p.S, tC.cpu().numpy())
    assert float(loss.item()) / Bsz == pytest.approx(lo, rel=1e-2)
    # against the FP64 network, which keeps activations exact where the device
    # stores BF16: storage can flip a ReLU mask, which adds terms the exact
    # network does not have, so this comparison is per parameter block (3e-2
    # of its norm)
    off = 0
    for (o, i) in M.shapes(p.n_out):
        for size in (o * i, o):
            a, b = g_gpu[off:off + size], g_ref[off:off + size]
            assert np.linalg.norm(a - b) <= 3e-2 * np.linalg.norm(b) + 1e-7, (off, np.linalg.norm(a - b),
                                                                              np.linalg.norm(b))
            off += size
    # element by element against the FP64 reference that rounds to BF16 where
    # the device does, with all three heads: what is left is FP32 accumulation
    # and the rare value whose FP32 and FP64 forms straddle a BF16 rounding
    # boundary (one BF16 step, 2^-8, of one term of a sum): every parameter
    # within 8e-3 of its gradient's absolute-value scale
    layers, k = [], 0
    for (o, i) in M.shapes(p.n_out):
        layers.append((w_bf[k:k + o * i].reshape(o, i), w_f[k + o * i:k + o * i + o]))
        k += o * i + o
    lo2, g_rnd, g_abs = _device_rounded_grads(layers, X.float().cpu().numpy().astype(np.float64), tA.cpu().numpy(),
                                              tB.cpu().numpy(), p.nA, p.nB, p.n_out, p.nC, p.S, tC.cpu().numpy())
    assert float(loss.item()) / Bsz == pytest.approx(lo2, rel=1e-4)
    err = np.abs(g_gpu - g_rnd)
    bound = 8e-3 * g_abs + 1e-7
    worst = int(np.argmax(err / bound))
    assert np.all(err <= bound), (worst, g_gpu[worst], g_rnd[worst], g_abs[worst],
                                  float((err / (g_abs + 1e-30)).max()))


def test_training_learns_the_first_passage_distribution(proposal):
    p = proposal
    data = p.generate(400_000, seed=123)
    held = p.generate(32_768, seed=124, p0=10_000_000)
    before = p.mean_loss(held)
    p.train(data, iters=600, batch=4096, lr=2e-3)
    after = p.mean_loss(held)
    assert after < before - 1.0, (before, after)
    # exit-face marginal predicted vs empirical on held-out data
    X = held["X"][:8192].contiguous()
    logits = p.logits(X).cpu().numpy()[:, :p.nA].reshape(-1, 6, p.J)
    pr = np.exp(logits - logits.max(axis=(1, 2), keepdims=True))
    pr /= pr.sum(axis=(1, 2), keepdims=True)
    pred_face = pr.sum(axis=2).mean(axis=0)
    tA = held["tA"][:8192].cpu().numpy()
    emp = np.bincount(tA[tA >= 0] // p.J, minlength=6) / max(1, (tA >= 0).sum())
    assert 0.5 * np.abs(pred_face - emp).sum() < 0.05, (pred_face, emp)


@pytest.mark.parametrize("Bsz", [64, 192, 4096])
def test_tensor_core_forward_matches_fp64(proposal, Bsz):
    """Logits of the tcgen05 forward pass against an FP64 forward of the same
    BF16 weights and inputs (hidden activations rounded to BF16 as stored),
    on batches that leave the last 128-row tile partly empty."""
    p = proposal
    d = p.generate(Bsz, seed=5150 + Bsz)
    X = d["X"]
    z = p.logits(X).cpu().numpy().astype(np.float64)
    R.mlp_status(p.stream())
    wb = p.wb.float().cpu().numpy().astype(np.float64)
    wf = p.wf.cpu().numpy().astype(np.float64)
    layers, off = [], 0
    for (o, i) in M.shapes(p.n_out):
        W = wb[off:off + o * i].reshape(o, i)
        off += o * i
        b = wf[off:off + o]
        off += o
        layers.append((W, b))
    h = X.float().cpu().numpy().astype(np.float64)
    for l, (W, b) in enumerate(layers):
        h = h @ W.T + b
        if l < 3:
            h = torch.tensor(np.maximum(h, 0.0), dtype=torch.float32).to(torch.bfloat16).double().numpy()
    err = np.abs(z - h).max() / max(1.0, np.abs(h).max())
    assert err < 2e-3, err


def _bf16(x):
    return torch.tensor(np.asarray(x), dtype=torch.float32).to(torch.bfloat16).double().numpy()


def _device_rounded_grads(layers, X, tA, tB, nA, nB, n_out, nC=0, S=0, tC=None):
    """Loss and gradients in FP64 with BF16 rounding exactly where the device
    stores BF16: hidden activations, the logit gradient used in products, and
    the back-propagated gradients; bias gradients sum the unrounded values.
    Rows with a negative head-A target take no part (but count in the mean);
    head C, when present, is a softmax over the S logits of the target's slice.
    Also returns, per parameter, the scale of its gradient: the same backward
    pass in absolute values (|d|, |W|, |h|), which bounds how far rounding
    anywhere upstream can move it."""
    B = X.shape[0]
    hs = [X]
    for l, (W, b) in enumerate(layers[:3]):
        hs.append(_bf16(np.maximum(hs[-1] @ W.T + b, 0.0)))
    W4, b4 = layers[3]
    z = hs[3] @ W4.T + b4
    g = np.zeros_like(z)
    loss = 0.0
    for r in range(B):
        if tA[r] < 0:
            continue
        heads = [(0, nA, tA[r]), (nA, nA + nB, nA + tB[r])]
        if nC and tC is not None and tC[r] >= 0:
            lo = nA + nB + (tC[r] // S) * S
            heads.append((lo, lo + S, nA + nB + tC[r]))
        for lo, hi, t in heads:
            zz = z[r, lo:hi]
            m = zz.max()
            lse = m + np.log(np.exp(zz - m).sum())
            loss += lse - z[r, t]
            g[r, lo:hi] = np.exp(zz - lse)
            g[r, t] -= 1.0
    g /= B
    # the scale of each gradient is carried backwards in absolute values: a
    # value that is small by cancellation inside d @ W still carries the
    # rounding of the larger terms it cancelled
    grads = [None] * 4
    mags = [None] * 4
    gb = _bf16(g)
    grads[3] = (gb.T @ hs[3], g.sum(axis=0))
    mags[3] = (np.abs(gb).T @ np.abs(hs[3]), np.abs(g).sum(axis=0))
    d, da = gb, np.abs(gb)
    for l in (2, 1, 0):
        W_next = layers[l + 1][0]
        mask = hs[l + 1] > 0
        df = (d @ W_next) * mask
        dfa = (da @ np.abs(W_next)) * mask
        db = _bf16(df)
        grads[l] = (db.T @ hs[l], df.sum(axis=0))
        mags[l] = (dfa.T @ np.abs(hs[l]), dfa.sum(axis=0))
        d, da = db, dfa
    flat = lambda gs: np.concatenate([np.concatenate([gw.ravel(), gbias]) for gw, gbias in gs])
    return loss / B, flat(grads), flat(mags)


@pytest.mark.parametrize("n_out,nA,nB", [(64, 40, 16), (128, 96, 32), (320, 288, 32)])
def test_network_gradients_for_narrow_and_wide_heads(n_out, nA, nB):
    """Loss and gradients of random networks whose output layer is narrower
    than, equal to or wider than the hidden layers (the backward pass reuses
    its transposed copies across layers), against an FP64 reference that
    rounds to BF16 where the device stores BF16; what is left is FP32
    accumulation and the fast exponential."""
    B.build()
    rng = np.random.default_rng(n_out)
    n_par = R.mlp_param_count(n_out)
    wf = torch.tensor(rng.normal(0.0, 0.1, n_par).astype(np.float32), device="cuda")
    wb = torch.empty(n_par, dtype=torch.bfloat16, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    R.mlp_to_bf16(n_out, wf.data_ptr(), wb.data_ptr(), s)
    batch = 192
    X = torch.tensor(rng.normal(0.0, 1.0, (batch, 16)), dtype=torch.bfloat16, device="cuda")
    tA = torch.tensor(rng.integers(0, nA, batch), dtype=torch.int32, device="cuda")
    tB = torch.tensor(rng.integers(0, nB, batch), dtype=torch.int32, device="cuda")
    work = torch.empty(R.mlp_work_bytes(batch, n_out), dtype=torch.uint8, device="cuda")
    grad = torch.empty(n_par, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    R.mlp_loss_grad(n_out, nA, nB, wf.data_ptr(), wb.data_ptr(), X.data_ptr(), tA.data_ptr(), tB.data_ptr(), batch,
                    work.data_ptr(), grad.data_ptr(), loss.data_ptr(), s)
    R.mlp_status(s)
    wbf = wb.float().cpu().numpy().astype(np.float64)
    w64 = wf.cpu().numpy().astype(np.float64)
    layers, off = [], 0
    for (o, i) in M.shapes(n_out):
        W = wbf[off:off + o * i].reshape(o, i)
        off += o * i
        layers.append((W, w64[off:off + o]))
        off += o
    lo, g_ref, g_abs = _device_rounded_grads(layers, X.float().cpu().numpy().astype(np.float64), tA.cpu().numpy(),
                                             tB.cpu().numpy(), nA, nB, n_out)
    assert float(loss.item()) / batch == pytest.approx(lo, rel=1e-4)
    g = grad.cpu().numpy().astype(np.float64)
    # element by element: with BF16 rounding where the device rounds, what is
    # left is FP32 accumulation and the rare value that rounds to the other
    # BF16 neighbour (its FP32 and FP64 forms straddle a rounding boundary),
    # which moves one term of a sum by one BF16 step (2^-8 of it): 8e-3 of the
    # gradient's absolute-value scale allows two such steps in one parameter
    err = np.abs(g - g_ref)
    bound = 8e-3 * g_abs + 1e-7
    worst = int(np.argmax(err / bound))
    assert np.all(err <= bound), (n_out, worst, g[worst], g_ref[worst], g_abs[worst],
                                  float((err / (g_abs + 1e-30)).max()))
