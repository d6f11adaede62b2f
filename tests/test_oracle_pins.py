"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
a textbook special case (BGK at gamma = 1), an independent formulation written
here from the cascade relations of Sec. 5 (central-moment relaxation with
explicit binomial shifts), library routines (numpy inverse, QR), the Eq. 44
constraint with the E terms of Eqs. 26-28, and conservation laws.
"""
import itertools

import numpy as np
import pytest

import oracle as orc
import workloads as wl

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)
# Eq. 5 monomials, in the paper's order
MONO = [np.ones(9), EX, EY, EX**2 + EY**2, EX**2 - EY**2, EX * EY, EX**2 * EY, EX * EY**2, EX**2 * EY**2]
# raw moments in the oracle's order (kappa_0, x, y, xx, yy, xy, xxy, xyy, xxyy)
RAW = [np.ones(9), EX, EY, EX**2, EY**2, EX * EY, EX**2 * EY, EX * EY**2, EX**2 * EY**2]


def test_lattice_matches_table():
    ex, ey, w, opp = orc.lattice()
    assert np.array_equal(ex, EX) and np.array_equal(ey, EY)
    for a in range(9):
        assert ex[opp[a]] == -ex[a] and ey[opp[a]] == -ey[a]
    assert np.isclose(w.sum(), 1.0)


def test_weights_from_rest_equilibrium():
    """Inverse map of the u = 0 raw equilibrium (Eq. 15) gives the D2Q9 weights."""
    keq = orc.raw_equilibrium(1.0, 0.0, 0.0, 0.37)
    f = orc.pops_from_raw(keq)
    assert np.allclose(f, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, atol=1e-16)


def test_inverse_map_against_numpy_inverse():
    T = np.array(RAW)  # rows: moment, columns: alpha
    Tinv = np.linalg.inv(T)
    rng = np.random.default_rng(1)
    for _ in range(20):
        k = rng.normal(size=9)
        assert np.allclose(orc.pops_from_raw(k), Tinv @ k, atol=1e-13)
        f = rng.normal(size=9)
        assert np.allclose(orc.raw_moments(f), T @ f, atol=1e-13)


def test_K_is_gram_schmidt_of_eq5_monomials():
    """K columns: orthogonal, and span(K_0..K_j) = span(T_0..T_j) for every j."""
    K = orc.K_columns()
    G = K @ K.T
    assert np.allclose(G - np.diag(np.diag(G)), 0.0)
    for j in range(9):
        Tj = np.array(MONO[: j + 1]).T
        # K_j lies in the span of the first j+1 monomials
        coef, res, *_ = np.linalg.lstsq(Tj, K[j], rcond=None)
        assert np.allclose(Tj @ coef, K[j], atol=1e-12)
        # and has a non-zero component on monomial j
        q, _ = np.linalg.qr(np.array(MONO[:j]).T) if j else (np.zeros((9, 0)), None)
        resid = K[j] - q @ (q.T @ K[j])
        assert np.linalg.norm(resid) > 1e-6


def test_K_scaling_matches_eq4_factors_and_cascade():
    """Printed factors omega3/12, omega4/4, omega5/4 (Eq. 4) and the cascade
    coefficients of Sec. 5 (-6 u_y g3, -2 u_y g4, -8 u_x g5, -4 g6, -2 g3 in g8)."""
    K = orc.K_columns()
    dot = lambda a, b: float(np.dot(a, b))
    assert dot(K[3], EX**2 + EY**2) == 12
    assert dot(K[4], EX**2 - EY**2) == 4
    assert dot(K[5], EX * EY) == 4
    assert dot(K[6], EX**2 * EY) == -4
    assert dot(K[7], EX * EY**2) == -4
    assert dot(K[3], EX**2) == 6          # -6 u_y g3 in the xxy relation
    assert dot(K[4], EX**2) == 2          # -2 u_y g4
    assert dot(K[5], EX * EY) == 4        # -8 u_x g5 (= 2 u_x * 4)
    assert dot(K[8], EX**2 * EY**2) == 4
    assert dot(K[3], EX**2 * EY**2) == 8  # -2 g3 in g8
    # g0..g2 = 0 and K3..K8 orthogonal to 1, e_x, e_y: mass and momentum conserved
    for j in range(3, 9):
        for m in (np.ones(9), EX, EY):
            assert dot(K[j], m) == 0


def _central_from_raw(k, ux, uy):
    """Central moments about u from raw moments (binomial theorem), same order."""
    k0, kx, ky, kxx, kyy, kxy, kxxy, kxyy, kxxyy = k
    c = np.zeros(9)
    c[0] = k0
    c[1] = kx - ux * k0
    c[2] = ky - uy * k0
    c[3] = kxx - 2 * ux * kx + ux**2 * k0
    c[4] = kyy - 2 * uy * ky + uy**2 * k0
    c[5] = kxy - ux * ky - uy * kx + ux * uy * k0
    c[6] = kxxy - uy * kxx - 2 * ux * kxy + 2 * ux * uy * kx + ux**2 * ky - ux**2 * uy * k0
    c[7] = kxyy - ux * kyy - 2 * uy * kxy + 2 * ux * uy * ky + uy**2 * kx - uy**2 * ux * k0
    c[8] = (kxxyy - 2 * ux * kxyy - 2 * uy * kxxy + ux**2 * kyy + uy**2 * kxx + 4 * ux * uy * kxy
            - 2 * ux * uy**2 * kx - 2 * ux**2 * uy * ky + ux**2 * uy**2 * k0)
    return c


def _central_from_pops(f, ux, uy):
    cx, cy = EX - ux, EY - uy
    mons = [np.ones(9), cx, cy, cx**2, cy**2, cx * cy, cx**2 * cy, cx * cy**2, cx**2 * cy**2]
    return np.array([np.dot(m, f) for m in mons])


def _pops_from_central(c, ux, uy):
    """Solve for the populations with the given central moments (numpy solve)."""
    cx, cy = EX - ux, EY - uy
    Mc = np.array([np.ones(9), cx, cy, cx**2, cy**2, cx * cy, cx**2 * cy, cx * cy**2, cx**2 * cy**2])
    return np.linalg.solve(Mc, c)


def test_binomial_shift_helper():
    rng = np.random.default_rng(3)
    f = rng.uniform(0.01, 0.3, 9)
    ux, uy = 0.07, -0.04
    assert np.allclose(_central_from_raw(orc.raw_moments(f), ux, uy), _central_from_pops(f, ux, uy))


def _central_moment_relaxation(fbar, gamma, w, M, gi_mode):
    """Independent formulation (Sec. 5 text): every non-conserved central moment
    relaxes to its central equilibrium; the cascade relations are this statement
    rewritten through the binomial theorem."""
    rho = fbar.sum()
    ux, uy = np.dot(fbar, EX) / rho, np.dot(fbar, EY) / rho
    c = _central_from_pops(fbar, ux, uy)
    s3, d4, c5 = c[3] + c[4], c[3] - c[4], c[5]
    # central equilibria: raw second-order equilibria (Eq. 15) minus rho u_i u_j,
    # plus the extended-equilibrium terms M3..M5 (Eq. 32/33)
    eq_s3 = 2 * rho / 3 + rho * (ux**2 + uy**2) * (1 / gamma - 1) + M[0]
    eq_d4 = rho * (ux**2 - uy**2) * (1 / gamma - 1) + M[1]
    eq_c5 = rho * ux * uy * (1 / gamma - 1) + M[2]
    if gi_mode == orc.GI_UNCORRECTED:
        eq6, eq7 = 0.0, 0.0
    else:  # raw kappa_xxy^eq with the boxed 1/gamma^2 term, shifted to central
        eq6 = rho * ux**2 * uy * (1 / gamma**2 - 3 / gamma + 2)
        eq7 = rho * ux * uy**2 * (1 / gamma**2 - 3 / gamma + 2)
    eq8 = rho / 9
    s3 += w[3] * (eq_s3 - s3)
    d4 += w[4] * (eq_d4 - d4)
    c5 += w[5] * (eq_c5 - c5)
    c6 = c[6] + w[6] * (eq6 - c[6])
    c7 = c[7] + w[7] * (eq7 - c[7])
    c8 = c[8] + w[8] * (eq8 - c[8])
    cpost = np.array([c[0], c[1], c[2], 0.5 * (s3 + d4), 0.5 * (s3 - d4), c5, c6, c7, c8])
    return _pops_from_central(cpost, ux, uy)


@pytest.mark.parametrize("gi_mode", [orc.GI_UNCORRECTED, orc.GI_CUBIC_ONLY, orc.GI_FULL])
def test_cascade_equals_central_moment_relaxation(gi_mode):
    rng = np.random.default_rng(7)
    for _ in range(40):
        gamma = rng.uniform(0.2, 1.0)
        w = [0, 0, 0] + list(rng.uniform(0.3, 1.9, 6))
        ux, uy = rng.uniform(-0.1, 0.1, 2)
        feq = orc.pops_from_raw(orc.raw_equilibrium(1.0 + rng.uniform(-0.02, 0.02), ux, uy, gamma))
        fbar = feq * (1 + 0.05 * rng.normal(size=9))
        drx, dry = rng.normal(scale=1e-3, size=2)
        p = orc.make_params(8, 8, gamma, w, gi_mode=gi_mode)
        ft, gh, M, _ = orc.collide_cell(p, fbar, drx, dry)
        ref = _central_moment_relaxation(fbar, gamma, w, M, gi_mode)
        assert np.allclose(ft, ref, atol=2e-15, rtol=0), np.abs(ft - ref).max()
        if gi_mode != orc.GI_FULL:
            assert np.all(M == 0)


def _product_form_equilibrium(rho, ux, uy):
    """Textbook D2Q9 product-form equilibrium: rho psi_ex(ux) psi_ey(uy) with
    psi_0(u) = 2/3 - u^2, psi_{+-1}(u) = (1/3 + u^2 +- u)/2."""
    def psi(e, u):
        return 2 / 3 - u * u if e == 0 else 0.5 * (1 / 3 + u * u + e * u)
    return np.array([rho * psi(EX[a], ux) * psi(EY[a], uy) for a in range(9)])


def test_gamma1_uncorrected_equal_rates_is_bgk():
    """gamma = 1, Eq. 4 kernel, all rates equal: the cascaded collision is BGK
    towards the product-form equilibrium (machine precision)."""
    rng = np.random.default_rng(11)
    for _ in range(30):
        om = rng.uniform(0.3, 1.9)
        p = orc.make_params(8, 8, 1.0, [0, 0, 0] + [om] * 6, gi_mode=orc.GI_UNCORRECTED)
        fbar = rng.uniform(0.01, 0.4, 9)
        fbar[0] += 0.4
        rho = fbar.sum()
        ux, uy = np.dot(fbar, EX) / rho, np.dot(fbar, EY) / rho
        bgk = fbar + om * (_product_form_equilibrium(rho, ux, uy) - fbar)
        ft, *_ = orc.collide_cell(p, fbar)
        assert np.allclose(ft, bgk, atol=1e-15, rtol=0)
        # CUBIC_ONLY coincides with Eq. 4 at gamma = 1 ((3/g - 1/g^2) = 2)
        p2 = orc.make_params(8, 8, 1.0, [0, 0, 0] + [om] * 6, gi_mode=orc.GI_CUBIC_ONLY)
        ft2, *_ = orc.collide_cell(p2, fbar)
        assert np.allclose(ft2, bgk, atol=1e-15, rtol=0)


def test_equilibrium_init_is_fixed_point_of_collision():
    """The Eq. 15 equilibrium (kernel-consistent fourth moment) is left unchanged
    by the Sec. 5 collision when there are no gradients.  The Eq. 4 kernel relaxes
    the third-order central moments to 0 instead of the boxed gamma^2 value, so for
    it the Eq. 15 state is a fixed point only at gamma = 1."""
    rng = np.random.default_rng(5)
    for gi_mode in (0, 1, 2):
        for _ in range(10):
            g = 1.0 if gi_mode == orc.GI_UNCORRECTED else rng.uniform(0.2, 1.0)
            ux, uy = rng.uniform(-0.1, 0.1, 2)
            feq = orc.pops_from_raw(orc.raw_equilibrium(1.02, ux, uy, g))
            w = [0, 0, 0] + list(rng.uniform(0.3, 1.9, 6))
            p = orc.make_params(8, 8, g, w, gi_mode=gi_mode)
            ft, gh, M, _ = orc.collide_cell(p, feq)
            assert np.allclose(ft, feq, atol=2e-16)


def test_gi_coefficients_satisfy_eq44_constraints():
    """(1 - w_j/2)(E_grho^j + E_gu^j) + m_j^eq(1) = 0 (Eq. 44) with the error terms
    of Eqs. 26-28 typed here independently of Eqs. 45-47."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        g = rng.uniform(0.1, 1.0)
        rho = rng.uniform(0.9, 1.1)
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        w3, w4, w5 = rng.uniform(0.2, 1.9, 3)
        dux, duy, drx, dry = rng.normal(size=4)
        a1 = 4 / g**2 - 1 / g
        b1 = 1 / g**2 - 1 / g
        cg = 1 / g - 1
        E3 = (2 / (3 * w3) * cg * (ux * drx + uy * dry)
              + rho / w3 * ((a1 * ux**2 + b1 * uy**2) * dux + (a1 * uy**2 + b1 * ux**2) * duy))
        E4 = (2 / (3 * w4) * cg * (ux * drx - uy * dry)
              + rho / w4 * ((a1 * ux**2 - b1 * uy**2) * dux + (-a1 * uy**2 + b1 * ux**2) * duy))
        E5 = (1 / (3 * w5) * cg * (ux * dry + uy * drx)
              + rho / w5 * b1 * ux * uy * (dux + duy))
        c = orc.gi_coefficients(rho, ux, uy, g, w3, w4, w5)
        M3 = c[0] * dux + c[1] * duy + c[2] * drx + c[3] * dry
        M4 = c[4] * dux - c[5] * duy + c[6] * drx - c[7] * dry
        M5 = c[8] * dux + c[9] * duy + c[10] * drx + c[11] * dry
        assert abs((1 - w3 / 2) * E3 + M3) < 1e-11 * (1 + abs(M3))
        assert abs((1 - w4 / 2) * E4 + M4) < 1e-11 * (1 + abs(M4))
        assert abs((1 - w5 / 2) * E5 + M5) < 1e-11 * (1 + abs(M5))


def test_gamma1_limit_matches_geier_dellar_form():
    """At gamma = 1: theta3_x = -3 rho (1/w3 - 1/2) ux^2, theta3_y likewise with uy,
    theta4_x = -3 rho (1/w4 - 1/2) ux^2, theta4_y = -3 rho (1/w4 - 1/2) uy^2, all
    other coefficients zero (the special case stated after Eq. 47)."""
    rho, ux, uy, w3, w4, w5 = 1.03, 0.08, -0.05, 1.2, 0.8, 0.8
    c = orc.gi_coefficients(rho, ux, uy, 1.0, w3, w4, w5)
    k3, k4 = 1 / w3 - 0.5, 1 / w4 - 0.5
    assert np.isclose(c[0], -3 * rho * k3 * ux**2)
    assert np.isclose(c[1], -3 * rho * k3 * uy**2)
    assert np.isclose(c[4], -3 * rho * k4 * ux**2)
    assert np.isclose(c[5], -3 * rho * k4 * uy**2)
    for i in (2, 3, 6, 7, 8, 9, 10, 11):
        assert c[i] == 0.0


def test_strain_solve_satisfies_eq51_eq52():
    """The returned strain rates solve Eqs. 51-52 (this pins the corrected sign of
    Eq. 55b: the printed form fails this back-substitution)."""
    rng = np.random.default_rng(4)
    for _ in range(50):
        g = rng.uniform(0.2, 1.0)
        rho = rng.uniform(0.95, 1.05)
        ux, uy = rng.uniform(-0.1, 0.1, 2)
        w3, w4 = rng.uniform(0.4, 1.9, 2)
        m3, m4, drx, dry = rng.normal(scale=1e-3, size=4)
        dux, duy, guarded = orc.strain_rates(rho, ux, uy, g, w3, w4, m3, m4, drx, dry)
        A, B, C = 4 / g**2 - 1 / g, 1 / g**2 - 1 / g, 1 / g - 1
        c1 = (2 / (3 * w3) - 0.5 * (A * ux**2 + B * uy**2)) * rho
        c2 = (2 / (3 * w3) - 0.5 * (A * uy**2 + B * ux**2)) * rho
        c1t = (2 / (3 * w4) - 0.5 * (A * ux**2 - B * uy**2)) * rho
        c2t = (2 / (3 * w4) - 0.5 * (A * uy**2 - B * ux**2)) * rho
        er = C / 3 * (ux * drx + uy * dry)
        ert = C / 3 * (ux * drx - uy * dry)
        assert np.isclose(-c1 * dux - c2 * duy, m3 - er, rtol=1e-12, atol=1e-18)
        assert np.isclose(-c1t * dux + c2t * duy, m4 - ert, rtol=1e-12, atol=1e-18)


def test_strain_solve_u0_closed_form():
    """u = 0: dux = -m3/(2a) - m4/(2b), duy = -m3/(2a) + m4/(2b), a = 2 rho/(3 w3),
    b = 2 rho/(3 w4)."""
    rho, w3, w4, m3, m4 = 1.01, 1.1, 0.7, 3e-4, -2e-4
    dux, duy, _ = orc.strain_rates(rho, 0.0, 0.0, 0.4, w3, w4, m3, m4, 0.01, -0.02)
    a, b = 2 * rho / (3 * w3), 2 * rho / (3 * w4)
    assert np.isclose(dux, -m3 / (2 * a) - m4 / (2 * b), rtol=1e-13)
    assert np.isclose(duy, -m3 / (2 * a) + m4 / (2 * b), rtol=1e-13)


def test_strain_solve_guard_reading():
    """The optional guard (the paper is silent on a vanishing determinant of
    Eqs. 51-52): it fires exactly when |D| < 0.1 |D0|, D from Eq. 53 and D0 its
    u = 0 value; then the solve is the u = 0 closed form applied to R3, R4 of
    Eq. 54 (the density-gradient terms stay); otherwise the guarded solve is the
    unguarded one."""
    rng = np.random.default_rng(12)
    fired = kept = 0
    for _ in range(4000):
        g = rng.uniform(0.15, 1.0)
        rho = rng.uniform(0.95, 1.05)
        ux, uy = rng.uniform(-0.3, 0.3, 2)
        w3, w4 = rng.uniform(0.4, 1.9, 2)
        m3, m4, drx, dry = rng.normal(scale=1e-3, size=4)
        A, B, C = 4 / g**2 - 1 / g, 1 / g**2 - 1 / g, 1 / g - 1
        a, b = 2 * rho / (3 * w3), 2 * rho / (3 * w4)
        c1 = a - 0.5 * rho * (A * ux**2 + B * uy**2)
        c2 = a - 0.5 * rho * (A * uy**2 + B * ux**2)
        c1t = b - 0.5 * rho * (A * ux**2 - B * uy**2)
        c2t = b - 0.5 * rho * (A * uy**2 - B * ux**2)
        D, D0 = -c1 * c2t - c1t * c2, -2 * a * b
        if abs(abs(D) - 0.1 * abs(D0)) < 1e-9 * abs(D0):
            continue  # too close to the threshold to call
        dux, duy, guarded = orc.strain_rates(rho, ux, uy, g, w3, w4, m3, m4, drx, dry, guard=True)
        assert guarded == (abs(D) < 0.1 * abs(D0))
        if guarded:
            fired += 1
            R3 = m3 - C / 3 * (ux * drx + uy * dry)
            R4 = m4 - C / 3 * (ux * drx - uy * dry)
            assert np.isclose(dux, -R3 / (2 * a) - R4 / (2 * b), rtol=1e-12, atol=1e-18)
            assert np.isclose(duy, -R3 / (2 * a) + R4 / (2 * b), rtol=1e-12, atol=1e-18)
        else:
            kept += 1
            assert (dux, duy) == orc.strain_rates(rho, ux, uy, g, w3, w4, m3, m4, drx, dry)[:2]
    assert fired > 20 and kept > 20, (fired, kept)


def test_strain_recovers_chapman_enskog_nonequilibrium():
    """A population set built with the Eq. 29/30 + Eq. 44 non-equilibrium part for a
    known strain returns that strain (m^(1) = -(2rho/3w)(div) + (w/2)E)."""
    rng = np.random.default_rng(9)
    for _ in range(20):
        g = rng.uniform(0.3, 1.0)
        rho = 1.0
        ux, uy = rng.uniform(-0.08, 0.08, 2)
        w3, w4 = rng.uniform(0.5, 1.8, 2)
        sxx, syy, drx, dry = rng.normal(scale=1e-3, size=4)
        A, B, C = 4 / g**2 - 1 / g, 1 / g**2 - 1 / g, 1 / g - 1
        E3 = (2 / (3 * w3) * C * (ux * drx + uy * dry)
              + rho / w3 * ((A * ux**2 + B * uy**2) * sxx + (A * uy**2 + B * ux**2) * syy))
        E4 = (2 / (3 * w4) * C * (ux * drx - uy * dry)
              + rho / w4 * ((A * ux**2 - B * uy**2) * sxx + (-A * uy**2 + B * ux**2) * syy))
        m3 = -2 * rho / (3 * w3) * (sxx + syy) + w3 / 2 * E3
        m4 = -2 * rho / (3 * w4) * (sxx - syy) + w4 / 2 * E4
        dux, duy, _ = orc.strain_rates(rho, ux, uy, g, w3, w4, m3, m4, drx, dry)
        assert np.isclose(dux, sxx, rtol=1e-10, atol=1e-16)
        assert np.isclose(duy, syy, rtol=1e-10, atol=1e-16)


def test_source_moments_are_moments_of_source():
    """S = T^-1 sigma' has zero mass and momentum F/gamma (so rho u = sum fbar e + F/2g)."""
    S = orc.pops_from_raw(orc.source_moments(1e-3, -2e-3, 0.05, 0.02, 0.4))
    assert abs(S.sum()) < 1e-18
    assert np.isclose(np.dot(S, EX), 1e-3 / 0.4) and np.isclose(np.dot(S, EY), -2e-3 / 0.4)


def test_source_moments_gamma1_are_the_shifted_first_order_source():
    """At gamma = 1 the raw source moments listed after Eq. 15 are those of the
    unpreconditioned cascaded forcing the paper builds on: a source whose
    central moments about u are (0, F_x, F_y) at orders 0 and 1 and zero at
    every higher order.  Computed here independently: the populations
    S = T^-1 sigma' are shifted to central moments about u by direct
    summation of (e - u)^m (e - u)^n, so a dropped factor or a wrong sign in
    any of sigma'_xx ... sigma'_xxyy leaves a nonzero higher central moment."""
    rng = np.random.default_rng(11)
    for _ in range(30):
        Fx, Fy = rng.uniform(-1e-3, 1e-3, 2)
        ux, uy = rng.uniform(-0.15, 0.15, 2)
        S = orc.pops_from_raw(orc.source_moments(Fx, Fy, ux, uy, 1.0))
        c = _central_from_pops(S, ux, uy)
        tol = 1e-14 * max(abs(Fx), abs(Fy))
        assert abs(c[0]) < tol
        assert abs(c[1] - Fx) < tol and abs(c[2] - Fy) < tol
        assert np.abs(c[3:]).max() < tol, c


def test_source_moments_gamma_scaling():
    """The preconditioning of the source moments stated after Eq. 15: the F_i
    terms (first order) carry 1/gamma, the F_i u_j terms (second order)
    1/gamma^2, and the third- and fourth-order moments are printed without a
    gamma.  Checked as ratios to the gamma = 1 moments, which the previous
    test fixes, for the nine components one by one."""
    rng = np.random.default_rng(12)
    power = np.array([0, 1, 1, 2, 2, 2, 0, 0, 0])
    for _ in range(30):
        Fx, Fy = rng.uniform(-1e-3, 1e-3, 2)
        ux, uy = rng.uniform(-0.15, 0.15, 2)
        g = rng.uniform(0.1, 1.0)
        s1 = orc.source_moments(Fx, Fy, ux, uy, 1.0)
        sg = orc.source_moments(Fx, Fy, ux, uy, g)
        assert sg[0] == 0.0 and s1[0] == 0.0
        assert np.allclose(sg[1:] * g ** power[1:], s1[1:], rtol=1e-13, atol=1e-22)


def _gradient(nx, ny, sides, fd, rho, solid=None):
    d = orc.Domain(nx, ny, 0.05, 0.5, sides, fd=fd, solid=solid)
    return d.density_gradient(rho)


def test_density_gradient_stencils_on_a_periodic_mode():
    """rho = 1 + a cos(kx) cos(qy) on a periodic box.  Central differences give
    d_x rho = -a sin k sin(kx) cos(qy) (and the mirror for y); the isotropic
    stencil 3 sum_a w_a e_a rho(x + e_a) named in Sec. 5 multiplies that by
    (2 + cos q) / 3, since its diagonal neighbours average over y +- 1."""
    nx, ny, a = 24, 20, 0.01
    k, q = 2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny
    x, y = np.arange(nx)[None, :], np.arange(ny)[:, None]
    rho = 1 + a * np.cos(k * x) * np.cos(q * y)
    ex = -a * np.sin(k) * np.sin(k * x) * np.cos(q * y)
    ey = -a * np.sin(q) * np.cos(k * x) * np.sin(q * y)
    gx, gy = _gradient(nx, ny, wl.periodic_sides(), orc.FD_CENTRAL, rho)
    assert np.abs(gx - ex).max() < 1e-16 and np.abs(gy - ey).max() < 1e-16
    gx, gy = _gradient(nx, ny, wl.periodic_sides(), orc.FD_ISOTROPIC, rho)
    assert np.abs(gx - ex * (2 + np.cos(q)) / 3).max() < 1e-16
    assert np.abs(gy - ey * (2 + np.cos(k)) / 3).max() < 1e-16


def test_density_gradient_ghost_rule():
    """rho = 1 + b x + c y.  Inside, both stencils are exact (b, c).  A missing
    neighbour (beyond a wall, or solid) takes the cell's own density: on the west
    wall both give d_x rho = b/2, while d_y rho is c (central) and 5c/6
    (isotropic: the two missing diagonals); at the south-west corner the
    isotropic stencil gives ((5b + c)/12, (5c + b)/12) and central (b/2, c/2); east
    of a lone solid cell the isotropic stencil gives (2b/3, c)."""
    nx, ny, b, c = 12, 10, 0.003, -0.002
    x, y = np.arange(nx)[None, :], np.arange(ny)[:, None]
    rho = 1 + b * x + c * y
    walls = ((wl.WALL, 0.0, 0.0),) * 4
    gxc, gyc = _gradient(nx, ny, walls, orc.FD_CENTRAL, rho)
    gxi, gyi = _gradient(nx, ny, walls, orc.FD_ISOTROPIC, rho)
    inner = (slice(1, ny - 1), slice(1, nx - 1))
    for g, v in ((gxc, b), (gyc, c), (gxi, b), (gyi, c)):
        assert np.allclose(g[inner], v, rtol=1e-12, atol=0)
    west = (slice(1, ny - 1), 0)
    assert np.allclose(gxc[west], b / 2, rtol=1e-12) and np.allclose(gyc[west], c, rtol=1e-12)
    assert np.allclose(gxi[west], b / 2, rtol=1e-12) and np.allclose(gyi[west], 5 * c / 6, rtol=1e-12)
    assert np.isclose(gxc[0, 0], b / 2, rtol=1e-12) and np.isclose(gyc[0, 0], c / 2, rtol=1e-12)
    assert np.isclose(gxi[0, 0], (5 * b + c) / 12, rtol=1e-12)
    assert np.isclose(gyi[0, 0], (5 * c + b) / 12, rtol=1e-12)
    solid = np.zeros((ny, nx), np.uint8)
    solid[5, 5] = 1
    gxs, gys = _gradient(nx, ny, walls, orc.FD_ISOTROPIC, rho, solid=solid)
    assert np.isclose(gxs[5, 6], 2 * b / 3, rtol=1e-12) and np.isclose(gys[5, 6], c, rtol=1e-12)
