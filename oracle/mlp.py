"""FP64 reference of the learned-proposal network (test infrastructure only).

16 inputs -> three hidden layers of 128 with ReLU -> n_out logits; head A is
a softmax over logits [0, nA), head B over [nA, nA + nB), and the optional
head C (nC = 6 S logits after head B) a conditional softmax: for a target
tC = f S + q only the S logits of slice f take part (the exit position on
face f given that face).  The loss is the batch mean of the heads'
cross-entropies (rows with target A < 0 are ignored, but still count in the
mean; a head-C target < 0 drops that head's term).  Parameters use the library's flat
layout: W1[128x16] b1 W2[128x128] b2 W3[128x128] b3 W4[n_out x 128] b4,
row-major W[out][in].
"""
import numpy as np

N_IN, N_HID = 16, 128


def shapes(n_out):
    return [(N_HID, N_IN), (N_HID, N_HID), (N_HID, N_HID), (n_out, N_HID)]


def unpack(flat, n_out):
    out, off = [], 0
    for (o, i) in shapes(n_out):
        W = np.asarray(flat[off:off + o * i], dtype=np.float64).reshape(o, i)
        off += o * i
        b = np.asarray(flat[off:off + o], dtype=np.float64)
        off += o
        out.append((W, b))
    return out


def pack(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def loss_and_grad(flat, n_out, nA, nB, X, tA, tB, nC=0, S=0, tC=None):
    """Mean loss over the batch and its gradient (flat, master layout)."""
    params = unpack(flat, n_out)
    X = np.asarray(X, dtype=np.float64)
    B = X.shape[0]
    acts = [X]
    for l, (W, b) in enumerate(params):
        z = acts[-1] @ W.T + b
        acts.append(np.maximum(z, 0.0) if l < 3 else z)
    logits = acts[-1]
    dlog = np.zeros_like(logits)
    loss = 0.0
    for r in range(B):
        if tA[r] < 0:
            continue
        heads = [(0, nA, tA[r]), (nA, nA + nB, nA + tB[r])]
        if nC and tC is not None and tC[r] >= 0:
            lo = nA + nB + (tC[r] // S) * S
            heads.append((lo, lo + S, nA + nB + tC[r]))
        for lo, hi, t in heads:
            z = logits[r, lo:hi]
            m = z.max()
            lse = m + np.log(np.exp(z - m).sum())
            loss += lse - logits[r, t]
            p = np.exp(z - lse)
            dlog[r, lo:hi] = p
            dlog[r, t] -= 1.0
    dlog /= B
    grads = [None] * 4
    d = dlog
    for l in range(3, -1, -1):
        W, b = params[l]
        grads[l] = (d.T @ acts[l], d.sum(axis=0))
        if l > 0:
            d = (d @ W) * (acts[l] > 0)
    return loss / B, pack(grads)
