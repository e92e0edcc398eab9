"""The library's host-side layout of a two-level mesh (hyb_two_level_layout; host memory, no
GPU) against the oracle's master / slave relations and its H (oracle/nonconforming.py): the
same multipliers one to one, the interface map W weight by weight, and H's sparsity pattern
exactly (Example 2.1; two multipliers couple when one element carries both)."""
import numpy as np
import pytest

from oracle.nonconforming import TwoLevelDiscretization
from paper_1801_08914_gb300 import inputs


@pytest.mark.parametrize("k,refine", [(0, True), (1, True), (2, True), (1, False)])
def test_layout_matches_the_oracle(k, refine):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1801_08914_gb300 import hyb
    nx, ny, nzc, nzf = 2, 3, 2, 1
    p = inputs.two_level_problem(nx, ny, nzc, nzf, k, 21, refine=refine, gamma=0.2)
    D = TwoLevelDiscretization(p)
    L = hyb.hyb_two_level_layout(nx, ny, nzc, nzf, k, refine)
    nfn, n, bI = (k + 1) ** 2, D.n, D.basis.n_interior
    assert L["n_lambda"] == D.n_lambda
    ef = L["elem_face"]
    assert ef.shape == (D.E, 6)

    def where(dof):
        e, loc = divmod(int(dof), n)
        f, m = divmod(loc - bI, nfn)
        return e, f, m

    # the oracle's multiplier r belongs to its slave dof: the library numbers it by the slave's face
    perm = np.empty(D.n_lambda, dtype=np.int64)
    for r_, (s, _) in enumerate(D.relations):
        e, f, m = where(s)
        assert ef[e, f] >= 0
        perm[r_] = ef[e, f] * nfn + m
    assert np.array_equal(np.sort(perm), np.arange(D.n_lambda))
    # boundary faces (no relation touches them) are -1
    used = {(where(s)[0], where(s)[1]) for s, _ in D.relations}
    used |= {(where(mm)[0], where(mm)[1]) for _, ms in D.relations for mm, _ in ms}
    for e in range(D.E):
        for f in range(6):
            assert (ef[e, f] >= 0) == ((e, f) in used), (e, f)
    if refine:
        seen = 0
        for s, ms in D.relations:
            e, f, m = where(s)
            if e < D.Ec or f != 4 or D.cell[e][3] != 0:
                continue
            _, i, j, _ = D.cell[e]
            sub = (i % 2) + 2 * (j % 2)
            ec = D.elem_index(0, i // 2, j // 2, p.nzc - 1)
            row = np.zeros(nfn)
            for mdof, w in ms:
                e2, f2, m2 = where(mdof)
                assert (e2, f2) == (ec, 5)
                row[m2] = w
            assert np.abs(L["W"][sub * nfn + m] - row).max() <= 1e-15
            assert ef[ec, 5] == ef[e, 4] - sub            # the coarse top face: first of its four
            seen += 1
        assert seen == 4 * nx * ny * nfn
    # pattern: multipliers of the rows of C that one element's columns reach
    C = D.C.tocsc()
    pat = set()
    for e in range(D.E):
        rr = perm[np.unique(C[:, e * n:(e + 1) * n].nonzero()[0])]
        pat.update((int(a), int(b)) for a in rr for b in rr)
    rp, col = L["row_ptr"], L["col"]
    assert rp[0] == 0 and rp[-1] == col.size
    lib_pat = set()
    for i in range(L["n_lambda"]):
        c = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0)
        lib_pat.update((i, int(x)) for x in c)
    assert lib_pat == pat
    H, _ = D.hybridize()
    big = np.abs(H) > 1e-13 * np.abs(H).max()
    for a, b in zip(*np.nonzero(big)):
        assert (int(perm[a]), int(perm[b])) in lib_pat


def test_layout_argument_errors():
    from paper_1801_08914_gb300 import hyb
    with pytest.raises(hyb.HybError):
        hyb.hyb_two_level_layout(0, 2, 1, 1, 1)
    with pytest.raises(hyb.HybError):
        hyb.hyb_two_level_layout(2, 2, 1, 1, 4)
