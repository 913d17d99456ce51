"""CPU checks of the arithmetic identities the CUDA pixel passes rely on.

The kernels do not enumerate active sets.  For a non-negative basis they
evaluate
    D_j = max(0, d_j),  d_j = (w_j.v - lambda) / G_jj,
    h_j = min(D_j, max(0, kappa (D_j - rho_j D_other))),
    rho_j = G12 / G_jj,  kappa = G11 G22 / det G,
with every quantity scaled by a power of two so that both max(0, .) become a
saturate; and count "h < lo" exactly as sat((lo - h) 2^K) with K = 24 - e for
lo in [2^e, 2^(e+1)).  These tests check both claims against the oracle's
enumeration and against exact comparisons."""
import numpy as np

from oracle import spcn_oracle as O


def closed_form(V, W, lam):
    G = W.T @ W
    det = G[0, 0] * G[1, 1] - G[0, 1] ** 2
    C = W.T @ V
    D1 = np.maximum((C[0] - lam) / G[0, 0], 0.0)
    D2 = np.maximum((C[1] - lam) / G[1, 1], 0.0)
    kap = G[0, 0] * G[1, 1] / det
    t1 = np.maximum(kap * (D1 - G[0, 1] / G[0, 0] * D2), 0.0)
    t2 = np.maximum(kap * (D2 - G[0, 1] / G[1, 1] * D1), 0.0)
    return np.vstack([np.minimum(D1, t1), np.minimum(D2, t2)])


def test_closed_form_equals_active_set_enumeration():
    rng = np.random.default_rng(1)
    for trial in range(300):
        W = rng.random((3, 2)) + 1e-3
        if trial % 2:
            W /= np.linalg.norm(W, axis=0)
        G = W.T @ W
        if G[0, 0] * G[1, 1] - G[0, 1] ** 2 < 1e-6:
            continue
        lam = [0.0, 0.1, 0.5][trial % 3]
        V = rng.normal(0.3, 1.0, size=(3, 2000))
        assert np.allclose(closed_form(V, W, lam), O.lasso2(V, W, lam), rtol=1e-10, atol=1e-10)


def test_closed_form_fails_for_negative_cross_term():
    # the identity needs G12 >= 0; with a negative entry it can be wrong,
    # which is why the library rejects negative bases
    W = np.array([[1.0, -0.8], [0.0, 0.6], [0.0, 0.0]])
    V = np.array([[0.2], [1.5], [0.0]])
    assert not np.allclose(closed_form(V, W, 0.1), O.lasso2(V, W, 0.1))


def test_saturated_below_count_is_exact():
    rng = np.random.default_rng(2)
    for _ in range(200):
        lo = np.float32(rng.uniform(1e-6, 0.9))
        e = int(np.floor(np.log2(lo)))
        K = 24 - e
        # values just below, at and above lo, and far away
        near = np.array([np.nextafter(lo, np.float32(0)), lo, np.nextafter(lo, np.float32(1))],
                        dtype=np.float32)
        h = np.concatenate([near, rng.uniform(0, 1, 500).astype(np.float32),
                            np.zeros(3, np.float32)])
        # fma(h, -2^K, lo 2^K) rounded once; float64 holds the exact product-sum here
        v = (-(2.0 ** K) * h.astype(np.float64) + float(lo) * 2.0 ** K).astype(np.float32)
        got = np.clip(v, 0, 1)
        assert np.array_equal(got, (h < lo).astype(np.float32))
