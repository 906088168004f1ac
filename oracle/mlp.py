"""FP64 oracle of the element-local MLP preconditioner (test infrastructure only).

The network is not in the paper; it is the learned right preconditioner layered
on the paper's method.  Plain numpy, FP64, written from the definitions:

  features of element K (din = 4*nb + 8):
      s   = sqrt(sum of r^2 over K and its face neighbours / (4*nb)) + 1e-30
      x   = [r_K, r_L0, r_L1, r_L2] / s            (zeros for a missing neighbour)
            + [log10(max(eps,1e-12))/6 + 1, b_x, b_y, alpha, J/sqrt(det J) (4 entries)]
  network g:  h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3),
              y  = W4 h3 + b4                       (width 128, y has nb entries)
  preconditioner:  z_K = A_KK^-1 (r_K + s * sigma * y_K)   (A_KK: diagonal block)
  training target for a residual r paired with its correction w (the
  one-layer-overlap patch solve):  t_K = (A_KK w_K - r_K) / s,
  sigma = RMS of all targets (fixed when training starts), and the network
  fits t / sigma: loss = mean over rows of 0.5 * |y - t/sigma|^2, Adam (beta1
  0.9, beta2 0.999, eps 1e-8, bias-corrected).

Parameters are one flat vector: W1 (128 x din, row-major), b1, W2, b2, W3, b3,
W4 (nb x 128), b4, sigma.
"""
import numpy as np

WIDTH = 128


NFEAT = 8


def din_of(nb):
    return 4 * nb + NFEAT


def sizes(nb):
    d = din_of(nb)
    return [(WIDTH, d), (WIDTH,), (WIDTH, WIDTH), (WIDTH,), (WIDTH, WIDTH), (WIDTH,), (nb, WIDTH), (nb,)]


def n_params(nb):
    return int(sum(np.prod(s) for s in sizes(nb))) + 1     # + sigma


def unpack(theta, nb):
    out, o = [], 0
    for s in sizes(nb):
        n = int(np.prod(s))
        out.append(theta[o:o + n].reshape(s))
        o += n
    return out


def features(r, nbr, nb, coef):
    """r [ne*nb]; nbr [ne,3] (-1 = none); coef [ne,8] = (eps, bx, by, alpha,
    J00, J01, J10, J11 scaled by 1/sqrt(det J)).  Returns X [ne, din], s [ne]."""
    ne = nbr.shape[0]
    R = r.reshape(ne, nb)
    P = np.zeros((ne, 4, nb))
    P[:, 0] = R
    for f in range(3):
        ok = nbr[:, f] >= 0
        P[ok, 1 + f] = R[nbr[ok, f]]
    s = np.sqrt((P ** 2).sum(axis=(1, 2)) / (4 * nb)) + 1e-30
    X = np.zeros((ne, din_of(nb)))
    X[:, :4 * nb] = P.reshape(ne, -1) / s[:, None]
    X[:, 4 * nb + 0] = np.log10(np.maximum(coef[:, 0], 1e-12)) / 6 + 1
    X[:, 4 * nb + 1] = coef[:, 1]
    X[:, 4 * nb + 2] = coef[:, 2]
    X[:, 4 * nb + 3] = coef[:, 3]
    X[:, 4 * nb + 4:4 * nb + 8] = coef[:, 4:8]
    return X, s


def forward(theta, X, nb):
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta, nb)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0)
    a3 = h2 @ W3.T + b3
    h3 = np.maximum(a3, 0)
    y = h3 @ W4.T + b4
    return y, (X, a1, h1, a2, h2, a3, h3)


def loss_and_grad(theta, X, T, nb):
    """Mean over rows of 0.5|y - t|^2 and its gradient (backpropagation)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta, nb)
    y, (X, a1, h1, a2, h2, a3, h3) = forward(theta, X, nb)
    n = X.shape[0]
    d = (y - T) / n
    loss = 0.5 * ((y - T) ** 2).sum() / n
    gW4 = d.T @ h3
    gb4 = d.sum(0)
    d3 = (d @ W4) * (a3 > 0)
    gW3 = d3.T @ h2
    gb3 = d3.sum(0)
    d2 = (d3 @ W3) * (a2 > 0)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (a1 > 0)
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4)] + [np.zeros(1)])
    return loss, g


def adam_step(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new theta, m, v."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def patch_correction(Ablk, nbr, r, nb):
    """One-layer-overlap patch correction w (the restricted additive Schwarz
    correction that the training targets are built from): for each element K,
    solve A_P w_P = r_P on the patch P = {K and its face neighbours} and keep
    w_K.  Ablk [ne,4,nb,nb]: slot 0 the diagonal block, slot 1+f the block
    coupling K to nbr[K,f]; nbr [ne,3] (-1 = no neighbour).  Dense numpy solve
    per patch."""
    ne = Ablk.shape[0]
    R = np.asarray(r, dtype=np.float64).reshape(ne, nb)
    w = np.zeros((ne, nb))
    for K in range(ne):
        E = [K] + [int(L) for L in nbr[K] if L >= 0]
        n = len(E) * nb
        AP = np.zeros((n, n))
        for p, Ep in enumerate(E):
            for q, Eq in enumerate(E):
                if p == q:
                    blk = Ablk[Ep, 0]
                else:
                    sl = [f for f in range(3) if nbr[Ep, f] == Eq]
                    if not sl:
                        continue
                    blk = Ablk[Ep, 1 + sl[0]]
                AP[p * nb:(p + 1) * nb, q * nb:(q + 1) * nb] = blk
        w[K] = np.linalg.solve(AP, np.concatenate([R[e] for e in E]))[:nb]
    return w.reshape(-1)


def target(Ablk, nbr, r, nb, s):
    """Training target t_K = (A_KK w_K - r_K) / s_K for the residual r."""
    ne = Ablk.shape[0]
    w = patch_correction(Ablk, nbr, r, nb).reshape(ne, nb)
    return (np.einsum("kij,kj->ki", Ablk[:, 0], w) - np.asarray(r).reshape(ne, nb)) / s[:, None]


def bf16_round_params(theta):
    """bf16-rounded weights with the f32 output scale left as is."""
    out = bf16_round(theta)
    out[-1] = np.float32(theta[-1])
    return out


def bf16_round(a):
    """Round to bfloat16 (nearest, ties to even) and back to float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
