"""Pins of the oracle's constrained global step (complementarity contact, Sec. 5.2):
the plain definition (sparse direct solve of the reduced system) agrees with the
paper's low-rank update written out densely (Alg. 4), with a dense solve of the
reduced matrix, and with the unconstrained solve when the contact set is empty."""
import numpy as np
import pytest

from oracle import contact
from oracle.model import Model
from oracle.pd_cpu import ScalarA
from workloads import small_beam


def _setup(seed):
    sc = small_beam(3, 2, 2, T=1, traction=False)
    L = ScalarA(Model(sc)).LA
    rng = np.random.default_rng(seed)
    nf = L.shape[0]
    b = rng.standard_normal((nf, 3))
    return L, b, rng, nf


@pytest.mark.parametrize("c", [1, 2, 5, 11])
def test_plain_definition_matches_woodbury_form(c):
    L, b, rng, nf = _setup(c)
    C = np.sort(rng.choice(nf, size=c, replace=False))
    xs = rng.standard_normal((c, 3))
    x = contact.constrained_solve(L, C, xs, b)
    xw = contact.woodbury_solve(L.toarray(), C, xs, b)
    assert np.allclose(x, xw, rtol=0, atol=1e-10 * np.abs(x).max())
    # a dense solve of the reduced matrix (another routine)
    keep = np.setdiff1d(np.arange(nf), C)
    xd = np.linalg.solve(L.toarray()[np.ix_(keep, keep)], b[keep])
    assert np.allclose(x[keep], xd, rtol=0, atol=1e-10 * np.abs(xd).max())
    assert np.array_equal(x[C], xs)


def test_empty_set_is_the_unconstrained_solve():
    L, b, rng, nf = _setup(7)
    x = contact.constrained_solve(L, np.zeros(0, dtype=np.int64), np.zeros((0, 3)), b)
    assert np.allclose(x, np.linalg.solve(L.toarray(), b), rtol=0, atol=1e-10 * np.abs(x).max())


def test_wrong_formula_is_detected():
    # a plausible slip (solving the full rows C' of A with x_C = x* instead of the
    # reduced block) gives a different answer, so the pins above can see it
    L, b, rng, nf = _setup(3)
    C = np.array([0, 5, 9])
    xs = rng.standard_normal((3, 3))
    keep = np.setdiff1d(np.arange(nf), C)
    Ld = L.toarray()
    wrong = np.linalg.solve(Ld[np.ix_(keep, keep)], b[keep] - Ld[np.ix_(keep, C)] @ xs)
    x = contact.constrained_solve(L, C, xs, b)
    assert not np.allclose(x[keep], wrong, atol=1e-8)
