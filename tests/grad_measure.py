"""Error measure for dL/dx of the differentiable normalisation (Eq. 1-4).

dL/dx_c = -(1/x_c) sum_k M_A[c,k] gv_k with gv_k = -gy_k y_k and M_A =
W_s G_AA^-1 diag(s) W_t^T restricted to the pixel's active set A (the chain
of Eq. 4, Eq. 3, the lasso of Eq. 2 and Eq. 1).  Where the three terms cancel,
|dL/dx_c| is far below the terms themselves, and no evaluation in a precision
with unit roundoff u can be closer to the exact value than about u times the
terms' magnitude.  The componentwise condition scale

    S_c = (|W_s| |G_AA^-1| diag(s) |W_t|^T |gy * y|)_c / x_c

is that magnitude (the same chain with every entry replaced by its absolute
value), and |computed - exact| <= tol * max(|exact|, S) is the componentwise
relative error bound used for FP32 against FP64 results."""
import numpy as np


def condition_scale(X, GY, Y, H, Ws, s, Wt):
    """S (3 x N) for float intensities X (3 x N), upstream gradient GY, the
    exact outputs Y, densities H (2 x N), source basis Ws, scale s and target
    basis Wt (all float64)."""
    G = Ws.T @ Ws
    Ginv = np.linalg.inv(G)
    a1, a2 = H[0] > 0, H[1] > 0
    gh = np.asarray(s)[:, None] * (np.abs(Wt.T) @ np.abs(GY * Y))
    gc = np.zeros_like(gh)
    both = a1 & a2
    gc[:, both] = np.abs(Ginv) @ gh[:, both]
    gc[0, a1 & ~a2] = gh[0, a1 & ~a2] / G[0, 0]
    gc[1, a2 & ~a1] = gh[1, a2 & ~a1] / G[1, 1]
    return (np.abs(Ws) @ gc) / np.maximum(X, 1.0)


def kkt_margin(X, H, Ws, i0s, lam, optical_density):
    """Per pixel, the distance of the lasso solution from an active-set change
    (the smallest |h_j| over active and |gradient_j| over inactive stains)."""
    V = optical_density(X.T, i0s).T
    g = (Ws.T @ Ws) @ H - Ws.T @ V + lam
    return np.min(np.abs(np.where(H > 0, H, g)), axis=0)
