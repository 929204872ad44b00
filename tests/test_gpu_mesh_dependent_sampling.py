"""Surrogate assembly driven by the mesh-dependent sampling length M(h) (Sec. 5.2,
Eq. MeshDependentSamplingLength) against the oracle.

M(h) comes from the C ABI (pinned to the oracle by the host-side tests), in the form of
the paper's 2-D experiment: M = max{1, floor(0.5 m^(1 - (p+1)/(q+1)))} with q = 5, i.e.
a = b = 1, C = 0.5, h = 1/m and a vanishing eps.  The sample indices are bit-exact and the
fields match the oracle surrogate built with the same M at 1e-12 of the largest entry, on
two meshes whose M(h) differ.
"""
import numpy as np
import pytest

from oracle.surrogate import mesh_dependent_sampling_length, sample_indices
from tests.oracle_cases import oracle_surrogate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_2004_05197_gb300 import iga
    from paper_2004_05197_gb300 import workloads as W

Q, A, B, C, EPS = 5, 1.0, 1.0, 0.5, 1e-9


def m_of_h(m, p):
    return iga.iga_sampling_length_for_mesh(1.0 / m, p, Q, A, B, C, EPS)


@pytest.mark.parametrize("n_el", [24, 60])
def test_mh_assembly_matches_oracle(n_el):
    p = 2
    m = n_el + p
    M = m_of_h(m, p)
    assert M == mesh_dependent_sampling_length(1.0 / m, p, Q, A, B, C, EPS)
    assert M == max(1, int(np.floor(0.5 * m ** (1.0 - (p + 1.0) / (Q + 1.0)))))
    w = W.scaled("annulus64_p2", n_el=n_el, q=Q, M=M)
    sp, S = oracle_surrogate(w)
    space = W.make_space(w)
    ops = iga.iga_surrogate_assemble(space, p, Q, M, 0)
    try:
        assert list(iga.iga_ops_sample_indices(ops)) == list(sample_indices(m, p, M))
        SK, SM = S.rows(sp.all_rows())
        t0 = (sp.D - 1) // 2
        info = iga.iga_ops_info_get(ops)
        for which, ref in ((iga.IGA_OP_K, SK[:, t0 + 1:].T), (iga.IGA_OP_M, SM[:, t0:].T)):
            nf = info.nK if which == iga.IGA_OP_K else info.nM
            t = torch.empty((nf, info.N), dtype=torch.float64, device="cuda")
            iga.iga_ops_copy_fields(ops, which, iga.IGA_F64, t)
            torch.cuda.synchronize()
            got = t.cpu().numpy()
            assert np.array_equal(got == 0.0, ref == 0.0)
            assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    finally:
        iga.iga_ops_destroy(ops)
        iga.iga_space_destroy(space)


def test_mh_grows_with_the_mesh():
    Ms = [m_of_h(n + 2, 2) for n in (24, 60, 96, 200, 400)]
    assert Ms == sorted(Ms) and Ms[-1] > Ms[0]
