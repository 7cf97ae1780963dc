"""Pin of the Gram decomposition the mixed-precision exact Galerkin uses
(Sec. 3, Phase 2 with the target's own operator, G = V_a^T A_i V_a).

With the five-point operator of Sec. 2.3 written as
    A v = cd v - c S v + qx o Dx v + qy o Dy v
(S v = v_E + v_W + v_N + v_S, Dx v = v_E - v_W, Dy v = v_N - v_S, zero
outside the grid; cd = 1/dt + 4c, c = g2/(2h^2), qx = f_x/(2h) - e (m_E -
m_W), qy likewise, e = g2/(8h^2)), the Gram matrix splits into a part of the
basis alone and a contraction of the target's coefficient rows with basis
products:
    G[p][q] = cd v_p.v_q - c v_p.S v_q + sum_k qx[k] v_p[k] (Dx v_q)[k]
                                       + sum_k qy[k] v_p[k] (Dy v_q)[k].
The test rebuilds G that way and checks it against V^T (A v_q) with the
oracle's own operator (coefficients and apply of the listing after Eq. 11),
for a grid with unequal sides, a drift field and a random lagged field: a
wrong sign, a swapped axis or a dropped boundary term fails it.
"""
import numpy as np


def _shift_ops(H, W):
    # point p = i*H + j (i along W: x, j along H: y), neighbours zero outside
    def nb(v):
        v2 = v.reshape(W, H)
        E = np.zeros_like(v2); E[:-1] = v2[1:]
        Wn = np.zeros_like(v2); Wn[1:] = v2[:-1]
        N = np.zeros_like(v2); N[:, :-1] = v2[:, 1:]
        S = np.zeros_like(v2); S[:, 1:] = v2[:, :-1]
        return E.ravel(), Wn.ravel(), N.ravel(), S.ravel()
    return nb


def test_gram_decomposition_matches_oracle_operator(orc):
    rng = np.random.default_rng(11)
    H, W = 7, 5
    N = H * W
    T, g2 = 1000, 0.37
    dt, h = 1.0 / T, 1.0 / H
    m = rng.uniform(0.1, 1.0, N)
    fx, fy = rng.normal(size=N), rng.normal(size=N)
    C = orc.coeffs(H, W, g2, dt, h, m, fx, fy)
    a = 6
    V = np.linalg.qr(rng.normal(size=(N, a)))[0].T          # a orthonormal rows
    G_ref = np.array([[V[p] @ orc.apply(H, W, C, V[q]) for q in range(a)] for p in range(a)])
    nb = _shift_ops(H, W)
    c = g2 / (2 * h * h)
    e = g2 / (8 * h * h)
    cd = 1.0 / dt + 4 * c
    mE, mW, mN, mS = nb(m)
    qx = fx / (2 * h) - e * (mE - mW)
    qy = fy / (2 * h) - e * (mN - mS)
    G = np.zeros((a, a))
    for q in range(a):
        vE, vW, vN, vS = nb(V[q])
        Sv, Dx, Dy = vE + vW + vN + vS, vE - vW, vN - vS
        for p in range(a):
            G[p, q] = cd * V[p] @ V[q] - c * V[p] @ Sv + qx @ (V[p] * Dx) + qy @ (V[p] * Dy)
    assert np.abs(G - G_ref).max() <= 1e-10 * np.abs(G_ref).max()
    # the target-dependent part is exactly the contraction Q . P over K = 2N
    Q = np.concatenate([qx, qy])
    P = np.array([[np.concatenate([V[p] * (nb(V[q])[0] - nb(V[q])[1]),
                                   V[p] * (nb(V[q])[2] - nb(V[q])[3])]) for q in range(a)] for p in range(a)])
    G0 = np.array([[cd * V[p] @ V[q] - c * V[p] @ sum(nb(V[q])) for q in range(a)] for p in range(a)])
    assert np.abs(G0 + P @ Q - G_ref).max() <= 1e-10 * np.abs(G_ref).max()
