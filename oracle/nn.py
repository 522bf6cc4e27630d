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
    (adaptive growth: t <- t + relu(conv3x3_dilation2(t, W_r) + b_r) for the
     extra blocks r = 1, 2, ... appended before the output layer)
    y   = conv3x3(t, W_out) + b_out                        C -> 1

conv3x3 with dilation d is the cross-correlation
    out[o, y, x] = bias[o] + sum_{c,ky,kx} W[o, c, ky, kx] in[c, y + d(ky-1), x + d(kx-1)]
with zeros outside the grid.  avgpool2 maps size s to floor(s/2) by the mean of
each 2x2 block.  Bilinear upsampling from m to n points per axis uses
half-pixel centres: src = (i + 0.5) m/n - 0.5 clamped below at 0, i0 = floor(src),
i1 = min(i0 + 1, m - 1), weight src - i0 on i1.

The 3D network (dim = 3, the variable-coefficient workload) is the same with
3x3x3 kernels, 2x2x2 average pooling (mean of each 2x2x2 block, down to 8^3)
and trilinear upsampling (the 1D interpolation applied along each axis).
Arrays are (C, n, n) in 2D and (C, n, n, n) in 3D, x the last axis.

Scaling (the paper leaves it open): the network sees u = b/s and is trained
towards x/s, s = rms(b); the guess is x0 = s * y.  Loss: the squared 2-norm of
Sec. 2.3 averaged over the batch and the grid points,
    L = 1/(B N) sum_b ||y_b - x_b/s_b||^2.
Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
theta -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
"""

import itertools
import math

import numpy as np

PARAM_ORDER_DOC = "in.w, in.b, level[0..L-1].w, level[l].b, dil.w, dil.b, out.w, out.b"


def level_sizes(n, min_size=8):
    sizes = [n]
    while sizes[-1] // 2 >= min_size:
        sizes.append(sizes[-1] // 2)
    return sizes


def param_shapes(n, C=32, dim=2, extra_blocks=0):
    """Ordered (name, shape) list of the network's parameters.  extra_blocks
    residual blocks res1, res2, ... (the adaptive growth of Sec. 2.1) come
    after out.b, so the base layout does not depend on them."""
    k = (3,) * dim
    shapes = [("in.w", (C, 1) + k), ("in.b", (C,))]
    for l in range(len(level_sizes(n))):
        shapes += [("level%d.w" % l, (C, C) + k), ("level%d.b" % l, (C,))]
    shapes += [("dil.w", (C, C) + k), ("dil.b", (C,)), ("out.w", (1, C) + k), ("out.b", (1,))]
    for r in range(1, extra_blocks + 1):
        shapes += [("res%d.w" % r, (C, C) + k), ("res%d.b" % r, (C,))]
    return shapes


def _blocks(params):
    """Residual blocks before the output layer, in order: dil, res1, res2, ..."""
    out = [("dil.w", "dil.b")]
    r = 1
    while ("res%d.w" % r) in params:
        out.append(("res%d.w" % r, "res%d.b" % r))
        r += 1
    return out


def _taps(dim):
    return list(itertools.product(range(3), repeat=dim))


def _window(pad, tap, d, size):
    return pad[(slice(None),) + tuple(slice(t * d, t * d + sz) for t, sz in zip(tap, size))]


def conv_fwd(inp, W, bias, d):
    """Cross-correlation with dilation d over the spatial axes of inp (C, ...),
    zeros outside the grid; W is (O, C, 3, ..., 3)."""
    size = inp.shape[1:]
    pad = np.zeros((inp.shape[0],) + tuple(sz + 2 * d for sz in size))
    pad[(slice(None),) + tuple(slice(d, d + sz) for sz in size)] = inp
    out = np.zeros((W.shape[0],) + size) + bias.reshape((-1,) + (1,) * len(size))
    for tap in _taps(len(size)):
        patch = _window(pad, tap, d, size)
        out += np.tensordot(W[(slice(None), slice(None)) + tap], patch, axes=([1], [0]))
    return out


def conv_bwd(inp, W, d, gout):
    """Returns (grad_in, grad_W, grad_bias) of conv_fwd for upstream gout."""
    size = inp.shape[1:]
    dim = len(size)
    pad = np.zeros((inp.shape[0],) + tuple(sz + 2 * d for sz in size))
    inner = (slice(None),) + tuple(slice(d, d + sz) for sz in size)
    pad[inner] = inp
    gpad = np.zeros_like(pad)
    gW = np.zeros_like(W)
    sp = tuple(range(1, dim + 1))
    for tap in _taps(dim):
        patch = _window(pad, tap, d, size)
        gW[(slice(None), slice(None)) + tap] = np.tensordot(gout, patch, axes=(sp, sp))
        win = (slice(None),) + tuple(slice(t * d, t * d + sz) for t, sz in zip(tap, size))
        gpad[win] += np.tensordot(W[(slice(None), slice(None)) + tap], gout, axes=([0], [0]))
    return gpad[inner], gW, gout.sum(axis=sp)


def avgpool2(x):
    """Mean of each 2x2 (2x2x2) block; size s -> floor(s/2) per axis."""
    dim = x.ndim - 1
    h = [sz // 2 for sz in x.shape[1:]]
    out = np.zeros((x.shape[0],) + tuple(h))
    for off in itertools.product(range(2), repeat=dim):
        out += x[(slice(None),) + tuple(slice(o, 2 * hh, 2) for o, hh in zip(off, h))]
    return out / 2 ** dim


def avgpool2_bwd(g, *size):
    dim = g.ndim - 1
    h = g.shape[1:]
    out = np.zeros((g.shape[0],) + tuple(size))
    for off in itertools.product(range(2), repeat=dim):
        out[(slice(None),) + tuple(slice(o, 2 * hh, 2) for o, hh in zip(off, h))] += g / 2 ** dim
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


def _along(U, x, axis):
    """Apply the matrix U (n x m) along spatial axis `axis` (1-based) of x."""
    return np.moveaxis(np.tensordot(U, x, axes=([1], [axis])), 0, axis)


def upsample(z, n):
    """Half-pixel (bi/tri)linear upsampling of z (C, m, ...) to n points per axis."""
    U = interp_matrix(z.shape[1], n)
    for ax in range(1, z.ndim):
        z = _along(U, z, ax)
    return z


def upsample_bwd(g, m):
    """Adjoint of upsample: g (C, n, ...) -> (C, m, ...)."""
    U = interp_matrix(m, g.shape[1]).T
    for ax in range(1, g.ndim):
        g = _along(U, g, ax)
    return g


def relu(x):
    return np.maximum(x, 0.0)


def forward(params, u, n, keep=False, dim=2):
    """params: dict name -> array; u: (n^dim,) normalised input.  Returns y
    (n^dim,) and, with keep=True, the activations needed by backward."""
    sizes = level_sizes(n)
    x = np.asarray(u, dtype=np.float64).reshape((1,) + (n,) * dim)
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
    # residual blocks t_{r+1} = t_r + relu(conv_dil2(t_r)), the first on t_0 = s
    t = s
    tins, preds = [], []
    for wn, bn in _blocks(params):
        pred = conv_fwd(t, params[wn], params[bn], 2)
        tins.append(t)
        preds.append(pred)
        t = t + relu(pred)
    y = conv_fwd(t, params["out.w"], params["out.b"], 1)
    if keep:
        return y.reshape(-1), dict(x=x, pre0=pre0, pools=pools, pres=pres, s=s, tins=tins,
                                   preds=preds, t=t)
    return y.reshape(-1)


def backward(params, cache, gy, n, dim=2):
    """Gradients of all parameters for upstream gradient gy (n^dim,)."""
    sizes = level_sizes(n)
    g = {}
    gy = np.asarray(gy, dtype=np.float64).reshape((1,) + (n,) * dim)
    gt, g["out.w"], g["out.b"] = conv_bwd(cache["t"], params["out.w"], 1, gy)
    blocks = _blocks(params)
    for r in range(len(blocks) - 1, -1, -1):
        wn, bn = blocks[r]
        gpred = gt * (cache["preds"][r] > 0)
        gin, g[wn], g[bn] = conv_bwd(cache["tins"][r], params[wn], 2, gpred)
        gt = gt + gin
    gs = gt
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
        acc = gpools[l - 1] + avgpool2_bwd(acc, *((sizes[l - 1],) * dim))
    ga0 = acc
    gpre0 = ga0 * (cache["pre0"] > 0)
    _, g["in.w"], g["in.b"] = conv_bwd(cache["x"], params["in.w"], 1, gpre0)
    return g


def loss_and_grads(params, inputs, targets, n, dim=2):
    """Batch MSE L = 1/(B N) sum ||y_b - target_b||^2 and its gradients.
    inputs / targets: (B, n^dim) normalised arrays."""
    B = len(inputs)
    N = n ** dim
    total = 0.0
    grads = {k: np.zeros_like(v) for k, v in params.items()}
    for b in range(B):
        y, cache = forward(params, inputs[b], n, keep=True, dim=dim)
        diff = y - np.asarray(targets[b], dtype=np.float64)
        total += float(diff @ diff)
        gb = backward(params, cache, 2.0 * diff / (B * N), n, dim=dim)
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
