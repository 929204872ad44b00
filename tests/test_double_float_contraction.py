"""The precision argument behind the band and sample-row quadratures' double-float
contractions (each value an unevaluated pair hi + lo of FP32 numbers, Dekker's product
with an FMA for the high parts, Knuth's TwoSum for the sums): the same pair arithmetic,
restated here in numpy FP32, contracts the 27 x 27 element stiffness of a 3-D p = 2
element (basis gradients of quadratic B-splines at 3^3 Gauss points, a random SPD metric
per point) within the parity bound the GPU fields are held to, 1e-12 |entry| +
1e-14 max|entry|, against the exactly rounded FP64 sum (math.fsum).  The GPU kernels are
pinned to the oracle separately (field parity tests)."""
import math

import numpy as np

f32 = np.float32


def split(x):
    hi = x.astype(f32)
    return hi, (x - hi.astype(np.float64)).astype(f32)


def two_sum(a, b):
    s = (a + b).astype(f32)
    bb = (s - a).astype(f32)
    return s, ((a - (s - bb).astype(f32)).astype(f32) + (b - bb).astype(f32)).astype(f32)


def mac(sh, sl, ah, al, bh, bl):
    p = (ah * bh).astype(f32)
    e = (ah.astype(np.float64) * bh.astype(np.float64) - p.astype(np.float64)).astype(f32)   # FMA residual
    e = (e + ((ah * bl).astype(f32) + (al * bh).astype(f32)).astype(f32)).astype(f32)
    s, t = two_sum(sh, p)
    t = (t + (sl + e).astype(f32)).astype(f32)
    h = (s + t).astype(f32)
    return h, (t - (h - s).astype(f32)).astype(f32)


def element_terms(rng):
    g = (np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)]) + 1.0) / 2.0
    gw = np.array([5.0, 8.0, 5.0]) / 18.0
    h = 1.0 / 96
    N = np.stack([(1 - g) ** 2 / 2, (-2 * g ** 2 + 2 * g + 1) / 2, g ** 2 / 2])
    dN = np.stack([-(1 - g), 1 - 2 * g, g]) / h
    A = rng.normal(size=(27, 3, 3)) * 0.1 + np.eye(3)
    G = np.einsum("qij,qkj->qik", A, A) * h ** 3
    grad = np.zeros((27, 27, 3))
    w = np.zeros(27)
    for q in range(27):
        q1, q2, q3 = q % 3, (q // 3) % 3, q // 9
        w[q] = gw[q1] * gw[q2] * gw[q3]
        for a in range(27):
            a1, a2, a3 = a % 3, (a // 3) % 3, a // 9
            grad[a, q] = [dN[a1, q1] * N[a2, q2] * N[a3, q3], N[a1, q1] * dN[a2, q2] * N[a3, q3],
                          N[a1, q1] * N[a2, q2] * dN[a3, q3]]
    Gg = np.einsum("qkl,aql->aqk", G, grad) * w[None, :, None]
    return Gg.reshape(27, 81), grad.reshape(27, 81)


def test_pair_contraction_meets_the_field_parity_bound():
    rng = np.random.default_rng(7)
    for _ in range(3):
        X, Y = element_terms(rng)                       # entry (a, b) = sum_t X[a, t] Y[b, t]
        exact = np.array([[math.fsum(X[a] * Y[b]) for b in range(27)] for a in range(27)])
        xh, xl = split(X)
        yh, yl = split(Y)
        sh = np.zeros((27, 27), dtype=f32)
        sl = np.zeros((27, 27), dtype=f32)
        for t in range(81):
            sh, sl = mac(sh, sl, xh[:, None, t], xl[:, None, t], yh[None, :, t], yl[None, :, t])
        got = sh.astype(np.float64) + sl.astype(np.float64)
        bound = 1e-12 * np.abs(exact) + 1e-14 * np.abs(exact).max()
        assert (np.abs(got - exact) <= 0.2 * bound).all()
        # plain FP32 would not do: its error is some 1e-7 of the largest entry
        plain = (X.astype(f32) @ Y.astype(f32).T).astype(np.float64)
        assert np.abs(plain - exact).max() > 1e-9 * np.abs(exact).max()
