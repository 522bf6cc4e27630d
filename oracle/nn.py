"""FP64 reference of the initial-guess network, its MSE loss, analytic
backward pass and the Adam update.

TEST INFRASTRUCTURE ONLY.

Architecture (a variation of the FluidNet pressure model, Sec. 2.1, Fig.
"Fluidnet": the input is average-pooled 2^d at a time while every resolution
is kept, each resolution goes through its own convolution, all are upsampled
back and summed, and output convolutions follow; the residual block after the
sum is the kind the paper stacks before the output layer, Fig. "Resblocks"):

    a0  = relu(conv3x3(u, W_in) + b_in)                    1 -> C channels
    p_0 = a0,  p_l = avgpool2(p_{l-1})  for sizes n, n/2, ... >= 8
    z_l = relu(conv3x3(p_l, W_l) + b_l)                    C -> C, one per level
    s   = sum_l upsample_bilinear(z_l -> n x n)
    t   = s + relu(conv3x3_dilation2(s, W_d) + b_d)        C -> C, residual
    y   = conv3x3(t, W_out) + b_out                        C -> 1

conv3x3 with dilation d is the cross-correlation
    out[o, y, x] = bias[o] + sum_{c,ky,kx} W[o, c, ky, kx] in[c, y + d(ky-1), x + d(kx-1)]
with zeros outside the grid.  avgpool2 maps size s to floor(s/2) by the mean of
each 2x2 block.  Bilinear upsampling from m to n points per axis uses
half-pixel centres: src = (i + 0.5) m/n - 0.5 clamped below at 0, i0 = floor(src),
i1 = min(i0 + 1, m - 1), weight src - i0 on i1.

Scaling (the paper leaves it open): the network sees u = b/s and is trained
towards x/s, s = rms(b); the guess is x0 = s * y.  Loss: the squared 2-norm of
Sec. 2.3 averaged over the batch and the grid points,
    L = 1/(B N) sum_b ||y_b - x_b/s_b||^2.
Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
theta -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
"""

import math

import numpy as np

PARAM_ORDER_DOC = "in.w, in.b, level[0..L-1].w, level[l].b, dil.w, dil.b, out.w, out.b"


def level_sizes(n, min_size=8):
    sizes = [n]
    while sizes[-1] // 2 >= min_size:
        sizes.append(sizes[-1] // 2)
    return sizes


def param_shapes(n, C=32):
    """Ordered (name, shape) list of the network's parameters."""
    shapes = [("in.w", (C, 1, 3, 3)), ("in.b", (C,))]
    for l in range(len(level_sizes(n))):
        shapes += [("level%d.w" % l, (C, C, 3, 3)), ("level%d.b" % l, (C,))]
    shapes += [("dil.w", (C, C, 3, 3)), ("dil.b", (C,)), ("out.w", (1, C, 3, 3)), ("out.b", (1,))]
    return shapes


def conv_fwd(inp, W, bias, d):
    C, H, Wd = inp.shape
    pad = np.zeros((C, H + 2 * d, Wd + 2 * d))
    pad[:, d:d + H, d:d + Wd] = inp
    out = np.zeros((W.shape[0], H, Wd)) + bias[:, None, None]
    for ky in range(3):
        for kx in range(3):
            patch = pad[:, ky * d:ky * d + H, kx * d:kx * d + Wd]
            out += np.einsum("oc,chw->ohw", W[:, :, ky, kx], patch)
    return out


def conv_bwd(inp, W, d, gout):
    """Returns (grad_in, grad_W, grad_bias) of conv_fwd for upstream gout."""
    C, H, Wd = inp.shape
    pad = np.zeros((C, H + 2 * d, Wd + 2 * d))
    pad[:, d:d + H, d:d + Wd] = inp
    gpad = np.zeros_like(pad)
    gW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            patch = pad[:, ky * d:ky * d + H, kx * d:kx * d + Wd]
            gW[:, :, ky, kx] = np.einsum("ohw,chw->oc", gout, patch)
            gpad[:, ky * d:ky * d + H, kx * d:kx * d + Wd] += np.einsum(
                "oc,ohw->chw", W[:, :, ky, kx], gout)
    return gpad[:, d:d + H, d:d + Wd], gW, gout.sum(axis=(1, 2))


def avgpool2(x):
    C, H, W = x.shape
    h, w = H // 2, W // 2
    return 0.25 * (x[:, 0:2 * h:2, 0:2 * w:2] + x[:, 1:2 * h:2, 0:2 * w:2]
                   + x[:, 0:2 * h:2, 1:2 * w:2] + x[:, 1:2 * h:2, 1:2 * w:2])


def avgpool2_bwd(g, H, W):
    C, h, w = g.shape
    out = np.zeros((C, H, W))
    for a in range(2):
        for b in range(2):
            out[:, a:2 * h:2, b:2 * w:2] += 0.25 * g
    return out


def interp_matrix(m, n):
    """(n x m) matrix of half-pixel bilinear interpolation from m to n points."""
    U = np.zeros((n, m))
    for i in range(n):
        src = (i + 0.5) * m / n - 0.5
        if src < 0.0:
            src = 0.0
        i0 = int(math.floor(src))
        if i0 > m - 1:
            i0 = m - 1
        i1 = min(i0 + 1, m - 1)
        lam = src - i0
        U[i, i0] += 1.0 - lam
        U[i, i1] += lam
    return U


def upsample(z, n):
    C, m, _ = z.shape
    U = interp_matrix(m, n)
    return np.einsum("im,cmk,jk->cij", U, z, U)


def upsample_bwd(g, m):
    C, n, _ = g.shape
    U = interp_matrix(m, n)
    return np.einsum("im,cij,jk->cmk", U, g, U)


def relu(x):
    return np.maximum(x, 0.0)


def forward(params, u, n, keep=False):
    """params: dict name -> array; u: (n*n,) normalised input.  Returns y (n*n,)
    and, with keep=True, the activations needed by backward."""
    sizes = level_sizes(n)
    x = np.asarray(u, dtype=np.float64).reshape(1, n, n)
    pre0 = conv_fwd(x, params["in.w"], params["in.b"], 1)
    a0 = relu(pre0)
    pools = [a0]
    for l in range(1, len(sizes)):
        pools.append(avgpool2(pools[-1]))
    pres = []
    s = np.zeros_like(a0)
    for l in range(len(sizes)):
        pre = conv_fwd(pools[l], params["level%d.w" % l], params["level%d.b" % l], 1)
        pres.append(pre)
        z = relu(pre)
        s = s + (z if l == 0 else upsample(z, n))
    pred = conv_fwd(s, params["dil.w"], params["dil.b"], 2)
    t = s + relu(pred)
    y = conv_fwd(t, params["out.w"], params["out.b"], 1)
    if keep:
        return y.reshape(-1), dict(x=x, pre0=pre0, pools=pools, pres=pres, s=s, pred=pred, t=t)
    return y.reshape(-1)


def backward(params, cache, gy, n):
    """Gradients of all parameters for upstream gradient gy (n*n,)."""
    sizes = level_sizes(n)
    g = {}
    gy = np.asarray(gy, dtype=np.float64).reshape(1, n, n)
    gt, g["out.w"], g["out.b"] = conv_bwd(cache["t"], params["out.w"], 1, gy)
    gpred = gt * (cache["pred"] > 0)
    gs_d, g["dil.w"], g["dil.b"] = conv_bwd(cache["s"], params["dil.w"], 2, gpred)
    gs = gt + gs_d
    gpools = [None] * len(sizes)
    for l in range(len(sizes)):
        gz = gs if l == 0 else upsample_bwd(gs, sizes[l])
        gpre = gz * (cache["pres"][l] > 0)
        gp, g["level%d.w" % l], g["level%d.b" % l] = conv_bwd(
            cache["pools"][l], params["level%d.w" % l], 1, gpre)
        gpools[l] = gp
    # pooling chain: p_l = avgpool2(p_{l-1}); accumulate from the coarsest level
    acc = gpools[-1]
    for l in range(len(sizes) - 1, 0, -1):
        acc = gpools[l - 1] + avgpool2_bwd(acc, sizes[l - 1], sizes[l - 1])
    ga0 = acc
    gpre0 = ga0 * (cache["pre0"] > 0)
    _, g["in.w"], g["in.b"] = conv_bwd(cache["x"], params["in.w"], 1, gpre0)
    return g


def loss_and_grads(params, inputs, targets, n):
    """Batch MSE L = 1/(B N) sum ||y_b - target_b||^2 and its gradients.
    inputs / targets: (B, n*n) normalised arrays."""
    B = len(inputs)
    N = n * n
    total = 0.0
    grads = {k: np.zeros_like(v) for k, v in params.items()}
    for b in range(B):
        y, cache = forward(params, inputs[b], n, keep=True)
        diff = y - np.asarray(targets[b], dtype=np.float64)
        total += float(diff @ diff)
        gb = backward(params, cache, 2.0 * diff / (B * N), n)
        for k in grads:
            grads[k] += gb[k]
    return total / (B * N), grads


def adam_update(theta, m, v, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def rms(b):
    b = np.asarray(b, dtype=np.float64)
    return math.sqrt(float(b @ b) / len(b))
