"""Mesh-dependent sampling length M(h) (Sec. 5.2, Eq. MeshDependentSamplingLength):
the oracle against values worked out by hand, and the C-ABI host routine against
the oracle (host logic only, no device work)."""
import numpy as np
import pytest

from oracle.surrogate import mesh_dependent_sampling_length as M_of_h


def test_worked_values():
    # p = 2, q = 3, a = b = 0, eps = 1/3: exponent 1/3 - 1 + 2/3 = 0, so M = floor(C)
    assert M_of_h(0.01, 2, 3, eps=1.0 / 3.0, C=5.5) == 5
    # p = 1, q = 3, b = 1, eps = 1/2: exponent -1/2 + 1/4 = -1/4; h = 1/16 gives h^-1/4 = 2
    assert M_of_h(1.0 / 16.0, 1, 3, b=1.0, eps=0.5, C=3.1) == 6
    # p = q = 2: exponent = eps > 0, so M(h) -> 1 as h -> 0 (no growth without q + b > p + a)
    assert M_of_h(1e-3, 2, 2, eps=0.2, C=3.0) == 1
    # the max{1, .} floor
    assert M_of_h(0.5, 2, 4, eps=0.1, C=0.1) == 1


def test_growth_and_consistency_order():
    """q + b > p + a and small eps: M(h) is non-decreasing as h -> 0 and
    H^(q+b) / h^(p+a) = (M h)^(q+b) / h^(p+a) -> 0."""
    p, q, eps, C = 2, 4, 0.1, 2.0
    hs = 1.0 / np.array([16, 32, 64, 128, 256, 512, 1024])
    Ms = [M_of_h(h, p, q, eps=eps, C=C) for h in hs]
    assert all(b >= a for a, b in zip(Ms, Ms[1:])) and Ms[-1] > Ms[0]
    ratio = [(M * h) ** q / h ** p for M, h in zip(Ms, hs)]
    assert ratio[-1] < ratio[0]


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        M_of_h(0.0, 2, 2)
    with pytest.raises(ValueError):
        M_of_h(0.1, 2, 2, eps=0.0)


def test_abi_matches_oracle():
    from paper_2004_05197_gb300 import build
    build.build()
    from paper_2004_05197_gb300 import iga
    cases = [(1.0 / n, p, q, a, b, C, eps) for n in (16, 40, 96, 300) for (p, q) in ((1, 2), (2, 3), (2, 4), (3, 5))
             for (a, b) in ((0.0, 0.0), (0.0, 1.0)) for (C, eps) in ((1.7, 0.05), (4.3, 0.2))]
    for h, p, q, a, b, C, eps in cases:
        want = M_of_h(h, p, q, a, b, C, eps)
        # stay away from exact integer boundaries, where FP64 pow may round either way
        x = C * h ** (eps - 1.0 + (p + a) / (q + b))
        if abs(x - round(x)) < 1e-9:
            continue
        assert iga.iga_sampling_length_for_mesh(h, p, q, a, b, C, eps) == want, (h, p, q, a, b, C, eps)
    with pytest.raises(iga.IgaError):
        iga.iga_sampling_length_for_mesh(-1.0, 2, 2)
