"""Pins of the oracle's lattice against the paper's printed coefficient table
and the isotropy identities of D3Q19 (Sec. 2 Method; Appendix coefficient
table; c_s^2 = 1/3 after Eq. LEQ)."""
import os
from fractions import Fraction

import numpy as np

import oracle
from oracle import lb_numpy, single_bgk

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "d3q19_coefficients.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        c2, mult, w, b = line.split()
        rows.append((int(c2), int(mult), Fraction(w), Fraction(b)))
    return rows


def test_velocity_set_is_d3q19():
    c, w, opp = oracle.lattice()
    assert c.shape == (19, 3)
    assert len({tuple(v) for v in c}) == 19
    c2 = (c * c).sum(axis=1)
    # rest + 6 at distance 1 + 12 at distance sqrt 2, no corners (sqrt 3)
    assert sorted(c2.tolist()) == [0] + [1] * 6 + [2] * 12
    assert np.abs(c).max() == 1
    # the same set as the independently enumerated numpy formulation
    assert {tuple(v) for v in c} == {tuple(v) for v in lb_numpy.VEL}
    assert {tuple(v) for v in c} == {tuple(v) for v in single_bgk.VELOCITIES}


def test_public_order_pairs_opposites():
    c, w, opp = oracle.lattice()
    assert (c[0] == 0).all()
    for i in range(1, 19):
        assert (c[opp[i]] == -c[i]).all()
        assert opp[i] == (i + 1 if i % 2 == 1 else i - 1)
    np.testing.assert_array_equal(c, lb_numpy.PUBLIC)


def test_weights_match_printed_table():
    c, w, _ = oracle.lattice()
    c2 = (c * c).sum(axis=1)
    for sq, mult, wt, _b in _golden_rows():
        sel = c2 == sq
        assert sel.sum() == mult
        np.testing.assert_allclose(w[sel], float(wt), rtol=0, atol=1e-17)


def test_isotropy_identities():
    c, w, _ = oracle.lattice()
    c = c.astype(np.float64)
    cs2 = 1.0 / 3.0
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(w @ c, 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, c, c), cs2 * np.eye(3), atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-16)
    d = np.eye(3)
    iso4 = cs2 * cs2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                        + np.einsum("ad,bc->abcd", d, d))
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso4, atol=1e-16)


def test_printed_perturbation_coefficients_satisfy_printed_constraints():
    """The B_i column of the same table obeys the isotropy constraints the
    Appendix states for it (sum B = 1/3, sum B c = 0, sum B c c = I/3); this
    checks the fixture was transcribed right."""
    c, _, _ = oracle.lattice()
    c2 = (c * c).sum(axis=1)
    bmap = {sq: b for sq, _m, _w, b in _golden_rows()}
    B = [bmap[int(s)] for s in c2]
    assert sum(B) == Fraction(1, 3)
    for a in range(3):
        assert sum(Bi * int(ci[a]) for Bi, ci in zip(B, c)) == 0
        for b in range(3):
            want = Fraction(1, 3) if a == b else Fraction(0)
            assert sum(Bi * int(ci[a]) * int(ci[b]) for Bi, ci in zip(B, c)) == want
