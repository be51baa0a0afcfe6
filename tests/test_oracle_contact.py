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


# ---------------------------------------------------------------- time step
import dataclasses  # noqa: E402

from oracle import newton  # noqa: E402
from workloads import contact_cube_c3  # noqa: E402


def _falling_cube(gap=0.002, vz=-0.6, N=3):
    sc = contact_cube_c3(N=N, T=4)
    x0 = sc.x0.copy()
    x0[:, 2] += gap - x0[:, 2].min()           # bottom face `gap` above the ground
    v0 = sc.v0 * 0.1
    v0[:, 2] += vz
    return dataclasses.replace(sc, x0=x0, v0=v0, k_contact=0.0, mu=0.0)


def test_step_in_flight_equals_newton():
    sc = _falling_cube(gap=0.05, vz=-0.1)
    model = Model(sc)
    x1, v1, info = contact.step_complementarity(model, sc.x0, sc.v0, sc.f_ext, sc.contact)
    assert info["C"].size == 0
    x2, v2, _ = newton.newton_step(model, sc.x0, sc.v0, sc.f_ext)
    assert np.allclose(x1, x2, rtol=0, atol=1e-12)


def test_contact_invariants():
    sc = _falling_cube()
    model = Model(sc)
    xs, vs, infos = contact.rollout_complementarity(model, sc.x0, sc.v0, sc.f_ext, sc.contact, 4)
    cand = np.flatnonzero(sc.contact)
    assert any(i["C"].size for i in infos)
    assert any("ray" in i["rules"] for i in infos)
    for t, i in enumerate(infos):
        x, y = xs[t + 1], i["y"]
        assert np.array_equal(x[i["C"]], i["xstar"])                  # held at the targets
        assert np.all(i["xstar"][:, 2] == 0.0)                          # targets on the ground
        assert i["rounds"] < 64                                         # the set settled
        free_set = ~np.isin(i["C"], i["locked"])                       # locked nodes may pull
        assert np.all(i["force"][free_set, 2] >= -i["tau_r"])          # pushing, never pulling
        assert np.all(x[np.setdiff1d(cand, i["C"]), 2] >= -i["tau_z"])  # no penetration
        # internal forces sum to zero: the contact forces carry the momentum change
        total = (model.m[:, None] * (x - y) / model.h ** 2).sum(axis=0)
        assert np.allclose(i["force"].sum(axis=0), total, rtol=1e-9, atol=1e-12 * np.abs(total).max())


def test_backward_matches_finite_differences():
    sc = _falling_cube()
    model = Model(sc)
    T = 3
    rng = np.random.default_rng(4)
    w = rng.standard_normal(sc.x0.shape)

    def run(x0, v0):
        xs, vs, infos = contact.rollout_complementarity(model, x0, v0, sc.f_ext, sc.contact, T)
        return float(np.sum(w * xs[-1])), xs, vs, infos

    L0, xs, vs, infos = run(sc.x0, sc.v0)
    gx = np.zeros_like(xs)
    gx[-1] = w
    g = contact.backward_complementarity(model, xs, vs, infos, gx)
    for key, base in (("g_v0", sc.v0), ("g_x0", sc.x0)):
        d = rng.standard_normal(base.shape)
        eps = 1e-7
        Lp, _, _, ip = run(*((sc.x0, sc.v0 + eps * d) if key == "g_v0" else (sc.x0 + eps * d, sc.v0)))
        Lm, _, _, im = run(*((sc.x0, sc.v0 - eps * d) if key == "g_v0" else (sc.x0 - eps * d, sc.v0)))
        for a, b in zip(ip, im):           # the contact sets do not change along the direction
            assert np.array_equal(a["C"], b["C"]) and a["rules"] == b["rules"]
        fd = (Lp - Lm) / (2 * eps)
        an = float(np.sum(g[key] * d))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-12), (key, fd, an)
