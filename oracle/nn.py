"""FP64 oracle of the learned preconditioner (test infrastructure only).

The workload statement (not the paper) asks for a small 3D convolutional
network on the active voxel grid that maps the Newton residual to a
correction used inside flexible CG.  The definition fixed here, written as
plain numpy on a dense node grid:

  x  = free * sqrt(D^-1) r / s,   s = RMS of sqrt(D^-1) r over free DOFs
  h1 = dof  * relu(conv(x,  W1))          3 -> 16 channels
  h2 = dof  * relu(conv(h1, W2))          16 -> 16
  y  = free * conv(h2, W3)                16 -> 3
  z  = D^-1 r + s sqrt(D^-1) y            (Jacobi plus the learned correction)

conv(a, W)[i] = sum_t W[t] @ a[i + d_t], t = (dz+1)*9 + (dy+1)*3 + (dx+1),
d_t = (dx, dy, dz) in {-1,0,1}^3, zero outside the grid; W has shape
(27, C_out, C_in).  No biases (the map is positively homogeneous).

Training loss for a residual / error pair (r, e = H^-1 r) of one Newton system H:
  L = 1 - z^T H e / sqrt(z^T H z * e^T H e) = 1 - z^T r / sqrt(z^T H z * r^T e)
one minus the H-cosine between the preconditioned residual z(r) and the error
(CG is invariant to the scale of the preconditioner, so only the direction of
z is scored; a z with z^T r <= 0 scores >= 1).  H enters as a callable.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
CHANNELS = (3, 16, 16, 3)


def conv3d(a, W):
    """a: (X, Y, Z, Cin) node grid; W: (27, Cout, Cin) -> (X, Y, Z, Cout)."""
    X, Y, Z, _ = a.shape
    out = np.zeros((X, Y, Z, W.shape[1]))
    pad = np.zeros((X + 2, Y + 2, Z + 2, a.shape[3]))
    pad[1:-1, 1:-1, 1:-1] = a
    for t, (dx, dy, dz) in enumerate(TAPS):
        sh = pad[1 + dx:1 + dx + X, 1 + dy:1 + dy + Y, 1 + dz:1 + dz + Z]
        out += sh @ W[t].T
    return out


def conv3d_backward(a, W, g):
    """Gradients of sum(g * conv3d(a, W)) w.r.t. a and W."""
    X, Y, Z, Cin = a.shape
    pad = np.zeros((X + 2, Y + 2, Z + 2, Cin))
    pad[1:-1, 1:-1, 1:-1] = a
    gpad = np.zeros_like(pad)
    gW = np.zeros_like(W)
    for t, (dx, dy, dz) in enumerate(TAPS):
        sl = (slice(1 + dx, 1 + dx + X), slice(1 + dy, 1 + dy + Y), slice(1 + dz, 1 + dz + Z))
        gW[t] = np.einsum("xyzo,xyzi->oi", g, pad[sl])
        gpad[sl] += g @ W[t]
    return gpad[1:-1, 1:-1, 1:-1], gW


def init_weights(seed=0, scale=None):
    """He-like seeded initialisation, float64, shapes (27, Cout, Cin)."""
    rng = np.random.default_rng(seed)
    Ws = []
    for l in range(3):
        cin, cout = CHANNELS[l], CHANNELS[l + 1]
        std = np.sqrt(2.0 / (27 * cin)) if scale is None else scale
        Ws.append(std * rng.standard_normal((27, cout, cin)))
    return Ws


def network(x, Ws, dof, free):
    """Forward pass; returns y and the activations needed by the backward pass."""
    p1 = conv3d(x, Ws[0])
    h1 = dof[..., None] * np.maximum(p1, 0.0)
    p2 = conv3d(h1, Ws[1])
    h2 = dof[..., None] * np.maximum(p2, 0.0)
    y = free[..., None] * conv3d(h2, Ws[2])
    return y, (x, p1, h1, p2, h2)


def network_backward(cache, gy, Ws, dof, free):
    x, p1, h1, p2, h2 = cache
    g3 = free[..., None] * gy
    gh2, gW3 = conv3d_backward(h2, Ws[2], g3)
    gp2 = gh2 * dof[..., None] * (p2 > 0)
    gh1, gW2 = conv3d_backward(h1, Ws[1], gp2)
    gp1 = gh1 * dof[..., None] * (p1 > 0)
    gx, gW1 = conv3d_backward(x, Ws[0], gp1)
    return [gW1, gW2, gW3], gx


def precondition(r, dinv, Ws, dof, free):
    """z = D^-1 r + s sqrt(D^-1) NN(sqrt(D^-1) r / s); r, dinv: (X, Y, Z, 3)."""
    sq = np.sqrt(dinv)
    u = sq * r
    nfree = max(int(free.sum()) * 3, 1)
    s = np.sqrt(np.sum(u * u) / nfree)
    z = dinv * r
    if s == 0:
        return z, None
    y, cache = network(u / s, Ws, dof, free)
    return z + s * sq * y, (cache, s, sq)


def loss_and_grad(r, e, dinv, Ws, dof, free, hvp):
    """Loss of one pair (one minus the H-cosine of z(r) and e) and its gradient w.r.t. the
    weights.  hvp: callable (X,Y,Z,3) -> (X,Y,Z,3), the Newton Hessian (masked)."""
    z, aux = precondition(r, dinv, Ws, dof, free)
    c = float(np.sum(e * hvp(e)))
    Hz = hvp(z)
    a = float(np.sum(z * r))
    b = float(np.sum(z * Hz))
    L = 1.0 - a / np.sqrt(b * c)
    if aux is None:
        return L, [np.zeros_like(W) for W in Ws]
    cache, s, sq = aux
    gz = -r / np.sqrt(b * c) + a * Hz / (np.sqrt(c) * b ** 1.5)
    gy = s * sq * gz
    gWs, _ = network_backward(cache, gy, Ws, dof, free)
    return L, gWs


def to_grid(values, ijk, shape):
    """Scatter key-ordered node values (n, C) at integer coords ijk into a dense grid."""
    out = np.zeros(tuple(shape) + (values.shape[1],))
    out[ijk[:, 0], ijk[:, 1], ijk[:, 2]] = values
    return out


def from_grid(grid, ijk):
    return grid[ijk[:, 0], ijk[:, 1], ijk[:, 2]]
