"""The angular fingerprint through spherical harmonics (the GPU's form for
angular order 6, sh_angular.cuh), written out in numpy FP64 from its
definition and checked against the oracle's pair sum (Sec. II.B, Eq. angular)
and, for its gradient, against central differences. This pins the identity
the kernel relies on:
  sum_{j != k} w_j w_k T_a(u_j . u_k) = sum_l b_al sum_m A_lm^2 - sum_j w_j^2,
A_lm = sum_j w_j Z_lm(u_j), with T_a = sum_l b_al P_l and the addition theorem
P_l(u . v) = sum_m Z_lm(u) Z_lm(v)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2107_11311_gb300 import inputs

L = 6
COMPS = [(l, m, kind) for m in range(L + 1) for l in range(m, L + 1) for kind in ((0,) if m == 0 else (0, 1))]
N2 = np.array([1.0 if m == 0 else 2.0 * math.factorial(l - m) / math.factorial(l + m) for (l, m, _) in COMPS])
LOF = np.array([l for (l, _, _) in COMPS])


def legendre_of_chebyshev(Ka):
    from numpy.polynomial import chebyshev as C, legendre as Lg
    b = np.zeros((Ka, L + 1))
    for a in range(Ka):
        c = Lg.poly2leg(C.cheb2poly([0] * a + [1]))
        b[a, :len(c)] = c
    return b


def components(u):
    """v_c(u) = Pbar_l^m(z) (C_m or S_m)(x, y) and its gradient in (x, y, z)."""
    x, y, z = u[:, 0], u[:, 1], u[:, 2]
    n = len(x)
    Cm, Sm = [np.ones(n)], [np.zeros(n)]
    for m in range(1, L + 1):
        Cm.append(x * Cm[-1] - y * Sm[-1])
        Sm.append(x * Sm[-1] + y * Cm[-2])
    P, dP = {}, {}
    for m in range(L + 1):
        P[(m, m)] = np.full(n, float(np.prod(np.arange(1, 2 * m, 2)))) if m else np.ones(n)
        dP[(m, m)] = np.zeros(n)
        if m + 1 <= L:
            P[(m + 1, m)] = (2 * m + 1) * z * P[(m, m)]
            dP[(m + 1, m)] = (2 * m + 1) * P[(m, m)]
        for l in range(m + 2, L + 1):
            a, b = (2 * l - 1) / (l - m), (l + m - 1) / (l - m)
            P[(l, m)] = a * z * P[(l - 1, m)] - b * P[(l - 2, m)]
            dP[(l, m)] = a * (P[(l - 1, m)] + z * dP[(l - 1, m)]) - b * dP[(l - 2, m)]
    v, g = np.zeros((len(COMPS), n)), np.zeros((len(COMPS), n, 3))
    for c, (l, m, kind) in enumerate(COMPS):
        T = Cm[m] if kind == 0 else Sm[m]
        if m:
            g[c, :, 0] = P[(l, m)] * m * (Cm[m - 1] if kind == 0 else Sm[m - 1])
            g[c, :, 1] = P[(l, m)] * m * (-Sm[m - 1] if kind == 0 else Cm[m - 1])
        v[c] = P[(l, m)] * T
        g[c, :, 2] = dP[(l, m)] * T
    return v, g


def fingerprint(d, s, rc, Ka):
    r = np.linalg.norm(d, axis=1)
    w = 0.5 * (np.cos(np.pi * r / rc) + 1.0)
    v, _ = components(d / r[:, None])
    b = legendre_of_chebyshev(Ka)
    out = []
    for wt in (w, s * w):
        A = v @ wt
        Q = np.zeros(L + 1)
        np.add.at(Q, LOF, N2 * A * A)
        out.append(b @ Q - np.sum(wt * wt))
    return out


def gradient(d, s, rc, Ka, g, gw):
    r = np.linalg.norm(d, axis=1)
    u = d / r[:, None]
    w = 0.5 * (np.cos(np.pi * r / rc) + 1.0)
    dw = -0.5 * np.pi / rc * np.sin(np.pi * r / rc)
    v, gv = components(u)
    b = legendre_of_chebyshev(Ka)
    A, B = v @ w, v @ (s * w)
    D, Dw = 2 * N2 * A * (g @ b)[LOF], 2 * N2 * B * (gw @ b)[LOF]
    out = np.zeros_like(d)
    for j in range(len(d)):
        k = D + s[j] * Dw
        E, F = k @ v[:, j], k @ gv[:, j, :]
        rad = dw[j] * (E - 2 * w[j] * (g.sum() + s[j] ** 2 * gw.sum()))
        out[j] = rad * u[j] + (w[j] / r[j]) * (F - (F @ u[j]) * u[j])
    return out


@pytest.fixture(scope="module")
def solid():
    st = inputs.amorphous(600, seed=9)
    m = inputs.make_model("amorphous")
    G = O.compute(m, st.pos, st.types, st.box, want_G=True, want_forces=False)["G"]
    return st, m, G, O.neighbour_lists(st.pos, st.box, m.rc_ang)


def _neigh(st, m, nl, i):
    d = np.array([st.pos[j] + np.array([nx, ny, nz]) * st.box - st.pos[i] for (j, nx, ny, nz) in nl[i]])
    s = np.asarray(m.type_weights)[st.types[[j for (j, _, _, _) in nl[i]]]]
    return d, s


def test_fingerprint_equals_the_pair_sum(solid):
    st, m, G, nl = solid
    Kr, Ka = m.order_rad + 1, m.order_ang + 1
    assert Ka - 1 == L
    for i in range(0, st.n, 37):
        d, s = _neigh(st, m, nl, i)
        plain, weighted = fingerprint(d, s, m.rc_ang, Ka)
        np.testing.assert_allclose(plain, G[i, Kr:Kr + Ka], rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(weighted, G[i, 2 * Kr + Ka:2 * Kr + 2 * Ka], rtol=1e-10, atol=1e-10)


def test_gradient_equals_central_differences(solid):
    st, m, _, nl = solid
    Ka = m.order_ang + 1
    rng = np.random.default_rng(3)
    for i in (5, 123):
        d, s = _neigh(st, m, nl, i)
        g, gw = rng.standard_normal(Ka), rng.standard_normal(Ka)
        an = gradient(d, s, m.rc_ang, Ka, g, gw)
        h = 1e-6
        for j in rng.choice(len(d), 4, replace=False):
            for a in range(3):
                dp, dm = d.copy(), d.copy()
                dp[j, a] += h
                dm[j, a] -= h
                Ep = sum(x @ y for x, y in zip((g, gw), fingerprint(dp, s, m.rc_ang, Ka)))
                Em = sum(x @ y for x, y in zip((g, gw), fingerprint(dm, s, m.rc_ang, Ka)))
                assert abs((Ep - Em) / (2 * h) - an[j, a]) <= 1e-6 * max(1.0, abs(an[j, a]))
