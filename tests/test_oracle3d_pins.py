"""Pins of the D3Q19 oracle (Section 2's scheme on the D3Q19 lattice) against what the lattice and
the mathematics fix: the lattice moments, the exact reduction to the (already pinned) D2Q9
oracle for fields invariant along any one axis, the uniform fixed point (Eq. 19), the uniform
transient, and mass conservation."""
import itertools

import numpy as np
import pytest

import oracle
import synth


def test_d3q19_lattice_moments():
    e, w = oracle.lattice3()
    assert len({tuple(v) for v in e}) == 19 and (np.abs(e).sum(axis=1) <= 2).all()
    assert {tuple(v) for v in e} == {tuple(-v) for v in e}
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(w @ e, 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("a,ai,aj->ij", w, e, e), np.eye(3) / 3.0, atol=1e-16)
    d = np.eye(3)
    iso = (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)) / 9.0
    np.testing.assert_allclose(np.einsum("a,ai,aj,ak,al->ijkl", w, e, e, e, e), iso, atol=1e-16)


def _run2d(k2, tau, nu, eps, g2, steps):
    p = oracle.Problem(tau, nu, eps, kappa=k2, g=g2)
    f = p.rest()
    p.run(f, steps)
    return p.fields(f)


def _run3d(k3, tau, nu, eps, g3, steps):
    p = oracle.Problem3D(tau, nu, eps, kappa=k3, g=g3)
    f = p.rest()
    p.run(f, steps)
    return p.fields(f)


@pytest.mark.parametrize("axis", ["z", "x", "y"])
def test_field_invariant_along_an_axis_reduces_to_d2q9(axis):
    """Summed over e along the invariant axis, the D3Q19 weights are the D2Q9 weights (4/9, 1/9,
    1/36), the equilibrium is linear in e . u and streaming along that axis moves nothing, so a
    field invariant along one axis, with no force along it, evolves like the D2Q9 problem on the
    other two axes: same rho and in-plane velocity, zero velocity along the axis."""
    k2 = synth.lognormal_kappa(12, 9, 2.5, 1.5, seed=51)          # [9][12]: 2-D (y, x)
    tau, nu, eps, steps = 0.8, 0.1, 0.9, 150
    g2 = (2e-6, -1.3e-6)
    r2, u2, v2 = _run2d(k2, tau, nu, eps, g2, steps)
    n = 3
    if axis == "z":       # 3-D (x, y) = 2-D (x, y)
        k3 = np.broadcast_to(k2[None, :, :], (n, 9, 12))
        r3, a3, b3, c3 = _run3d(k3, tau, nu, eps, (g2[0], g2[1], 0.0), steps)
        r3, a3, b3, c3 = (t[1] for t in (r3, a3, b3, c3))
    elif axis == "x":     # 3-D (y, z) = 2-D (x, y): kappa[z][y][x] = k2[z][y]
        k3 = np.broadcast_to(k2[:, :, None], (9, 12, n))
        r3, c3, a3, b3 = _run3d(k3, tau, nu, eps, (0.0, g2[0], g2[1]), steps)
        r3, a3, b3, c3 = (t[:, :, 1] for t in (r3, a3, b3, c3))
    else:                 # 3-D (x, z) = 2-D (x, y): kappa[z][y][x] = k2[z][x]
        k3 = np.broadcast_to(k2[:, None, :], (9, n, 12))
        r3, a3, c3, b3 = _run3d(k3, tau, nu, eps, (g2[0], 0.0, g2[1]), steps)
        r3, a3, b3, c3 = (t[:, 1, :] for t in (r3, a3, b3, c3))
    # both oracles store full f (~0.05 per population) while u ~ 1e-7: velocities agree to the
    # cancellation floor, ~1e-16 absolute (1e-9 of the velocity scale); a wrong weight, velocity or
    # stream direction shows up at order one
    scale = max(np.abs(u2).max(), np.abs(v2).max())
    np.testing.assert_allclose(r3, r2, rtol=0, atol=1e-14)
    np.testing.assert_allclose(a3, u2, rtol=0, atol=2e-9 * scale)
    np.testing.assert_allclose(b3, v2, rtol=0, atol=2e-9 * scale)
    assert np.abs(c3).max() <= 2e-9 * scale


def test_uniform_fixed_point_eq19_in_3d():
    """Eq. 19 in three dimensions: with uniform kappa, f_a = w_a rho0 (1 + 3 e_a . kappa G / nu)
    is a fixed point of the step."""
    e, w = oracle.lattice3()
    kap, nu, eps, tau = 3e-3, 0.05, 0.8, 0.7
    G = np.array([1e-6, -2e-6, 0.5e-6])
    p = oracle.Problem3D(tau, nu, eps, kappa=np.full((4, 3, 5), kap), g=G)
    u = kap * G / nu
    f = np.broadcast_to(w * (1.0 + 3.0 * (e @ u)), (4, 3, 5, 19)).copy()
    np.testing.assert_allclose(p.step(f), f, rtol=0, atol=1e-16)
    _, uu, vv, ww = p.fields(f)
    # j ~ 1e-7 is a sum of populations ~0.05 (the oracle stores full f): ~1e-15 absolute
    np.testing.assert_allclose([uu.mean(), vv.mean(), ww.mean()], u, rtol=0, atol=1e-14)


def test_uniform_transient_closed_form_in_3d():
    """Uniform state from rest: j' = (2 d - 1) j + d eps rho G with d = 1 / (1 + eps nu / (2 kappa))
    (any lattice; only the moments enter), and u = d (j + eps rho G / 2) / rho."""
    kap, nu, eps, tau = 2e-2, 0.1, 0.9, 0.6
    G = np.array([3e-6, 1e-6, -2e-6])
    p = oracle.Problem3D(tau, nu, eps, kappa=np.full((2, 3, 4), kap), g=G)
    f = p.rest()
    d = 1.0 / (1.0 + eps * nu / (2.0 * kap))
    j = np.zeros(3)
    for n in range(1, 40):
        f = p.step(f)
        j = (2 * d - 1) * j + d * eps * G
        _, uu, vv, ww = p.fields(f)
        np.testing.assert_allclose([uu[0, 0, 0], vv[0, 0, 0], ww[0, 0, 0]], d * (j + 0.5 * eps * G),
                                   rtol=0, atol=1e-15)         # cancellation in j, as above


def test_mass_conservation_and_symmetry_in_3d():
    rng = np.random.default_rng(52)
    kap = np.exp(rng.normal(-4.0, 1.5, (5, 6, 7)))
    kap[1, 2, 3] = 0.0
    kap[3, 1, 4] = np.inf
    p = oracle.Problem3D(0.9, 0.1, 0.8, kappa=kap, g=(1e-6, 2e-6, -1e-6))
    f = p.rest()
    p.run(f, 120)
    rho, u, v, w = p.fields(f)
    assert abs(rho.sum() - rho.size) <= 1e-12 * rho.size
    assert u[1, 2, 3] == 0.0 and v[1, 2, 3] == 0.0 and w[1, 2, 3] == 0.0   # blocked cell
    # mirror z -> -z (with gz -> -gz) mirrors the flow
    pm = oracle.Problem3D(0.9, 0.1, 0.8, kappa=kap[::-1].copy(), g=(1e-6, 2e-6, 1e-6))
    fm = pm.rest()
    pm.run(fm, 120)
    _, um, vm, wm = pm.fields(fm)
    s = np.abs(u).max()
    np.testing.assert_allclose(um[::-1], u, atol=1e-12 * s)
    np.testing.assert_allclose(wm[::-1], -w, atol=1e-12 * s)


# ------------------------------------------------- three-dimensional local problems (Eq. 17)

def test_local_keff3_uniform_cube_is_kappa_identity():
    r = oracle.local_keff3(np.full((5, 5, 5), 2e-3), 1.0, 1.0 / 6.0, 1.0, 1e-6, tol=1e-12, max_steps=100000)
    np.testing.assert_allclose(np.diag(r["keff"]), 2e-3, rtol=1e-9)
    # off-diagonals are rounding only: the cancellation floor of full-f storage, ~1e-10 of K*
    assert np.abs(r["keff"] - np.diag(np.diag(r["keff"]))).max() < 1e-9 * 2e-3


def test_local_keff3_of_a_z_invariant_cube_is_the_2d_local_keff():
    """The exact D3Q19 -> D2Q9 reduction of a field invariant along z: the xy block of K* is the
    2-D local K* of the slice (same stop rule, same step counts) and nothing couples to z."""
    k2 = synth.lognormal_kappa(6, 6, 2.0, 1.2, seed=55)
    r3 = oracle.local_keff3(np.broadcast_to(k2[None], (6, 6, 6)).copy(), 1.0, 1.0 / 6.0, 1.0, 1e-6,
                            tol=1e-9, max_steps=100000)
    r2 = oracle.local_keff(k2, 1.0, 1.0 / 6.0, 1.0, 1e-6, tol=1e-9, max_steps=100000)
    k2d = np.array([[r2["keff"][0], r2["keff"][1]], [r2["keff"][2], r2["keff"][3]]])
    assert r3["steps"][:2] == r2["steps"]
    np.testing.assert_allclose(r3["keff"][:2, :2], k2d, rtol=0, atol=1e-9 * np.abs(k2d).max())
    assert np.abs(r3["keff"][2, :2]).max() < 1e-9 * np.abs(k2d).max()    # rounding floor, as above
    assert np.abs(r3["keff"][:2, 2]).max() < 1e-9 * np.abs(k2d).max()


def test_local_keff3_axis_permutation():
    """Relabelling the axes of the cube (x, y, z) -> (y, z, x) permutes K* the same way."""
    rng = np.random.default_rng(56)
    k = np.exp(rng.normal(-5.0, 1.0, (4, 4, 4)))
    a = oracle.local_keff3(k, 1.0, 1.0 / 6.0, 1.0, 1e-6, tol=1e-11, max_steps=100000)["keff"]
    # new field K'[z'][y'][x'] with x' = y, y' = z, z' = x: K'[x][z][y] = K[z][y][x]
    kp = np.transpose(k, (2, 0, 1)).copy()
    b = oracle.local_keff3(kp, 1.0, 1.0 / 6.0, 1.0, 1e-6, tol=1e-11, max_steps=100000)["keff"]
    P = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]])        # new axis i is old axis perm[i]
    np.testing.assert_allclose(b, P @ a @ P.T, rtol=1e-7, atol=1e-9 * np.abs(a).max())


def test_local_keff3_parallel_layers_darcy_arithmetic_mean():
    """Table 2's setting in three dimensions: kappa varies along x in two bands, tau = 1/2 (Darcy);
    driven along y or z the flow sees the layers in parallel: K*_yy = K*_zz = arithmetic mean."""
    ex = synth.paper_experiment("E3", ratio=10.0, ny=1)
    k1, k2 = float(ex["kappa"][0, 0]), float(ex["kappa"][0, 10])
    cube = np.broadcast_to(np.array([k1] * 4 + [k2] * 4)[None, None, :], (8, 8, 8)).copy()
    r = oracle.local_keff3(cube, ex["tau"], ex["nu"], ex["eps"], 1e-6, tol=1e-11, max_steps=20000)
    mean = 0.5 * (k1 + k2)
    assert abs(r["keff"][1, 1] - mean) <= 2e-6 * mean and abs(r["keff"][2, 2] - mean) <= 2e-6 * mean


# ------------------------------------------------------------------ tensor K* (Eq. 18 in 3-D)

def _random_tensor_field(shape, seed):
    """Per-cell K* with a dominant positive diagonal and small, non-symmetric off-diagonals."""
    rng = np.random.default_rng(seed)
    K = np.zeros(shape + (3, 3))
    for i in range(3):
        K[..., i, i] = 1e-2 * np.exp(0.8 * rng.standard_normal(shape))
    off = 1.5e-3 * rng.standard_normal(shape + (3, 3))
    off[..., [0, 1, 2], [0, 1, 2]] = 0.0
    return K + off


def test_tensor_diagonal_is_the_scalar_run():
    """K* = kappa I in every cell is the scalar-kappa problem (Eq. 18 reduces to Eq. 6)."""
    k = synth.lognormal_kappa3d(5, 4, 6, 2.0, 1.5, seed=81).astype(np.float64)
    K = np.zeros(k.shape + (3, 3))
    for i in range(3):
        K[..., i, i] = k
    g = (1.5e-6, -1e-6, 0.7e-6)
    a = oracle.Problem3D(0.8, 0.1, 0.9, kappa=k, g=g)
    b = oracle.Problem3D(0.8, 0.1, 0.9, ktensor=K, g=g)
    fa, fb = a.rest(), b.rest()
    a.run(fa, 120)
    b.run(fb, 120)
    ua, ub = a.fields(fa), b.fields(fb)
    scale = max(np.abs(t).max() for t in ua[1:])
    for x, y in zip(ua[1:], ub[1:]):
        np.testing.assert_allclose(y, x, rtol=0, atol=1e-9 * scale)


def test_tensor_uniform_fixed_point_is_k_g_over_nu():
    """Eq. 18 with a uniform, non-symmetric K*: the uniform state f_a = w_a rho0 (1 + 3 e_a . u)
    with u = K* G / nu is a fixed point (then u_eq = u and (eps nu / 2) K*^-1 u = eps G / 2), and
    a run from rest converges to it. A transposed K* gives K*^T G and fails."""
    K0 = np.array([[2.0, 0.3, 0.1], [0.2, 1.5, 0.4], [0.05, 0.25, 1.2]]) * 1e-2
    nu, g = 0.1, np.array([1e-6, -2e-6, 0.5e-6])
    K = np.broadcast_to(K0, (2, 3, 2, 3, 3)).copy()
    p = oracle.Problem3D(1.0, nu, 0.7, ktensor=K, g=tuple(g))
    u = K0 @ g / nu
    e, w = oracle.lattice3()
    f = np.broadcast_to(w * (1.0 + 3.0 * (e @ u)), (2, 3, 2, 19)).copy()
    np.testing.assert_allclose(p.step(f), f, rtol=0, atol=2e-16)     # a few ulps of w_0 = 1/3
    # u ~ 1e-7 is recovered from full f ~ 0.05: the cancellation floor is ~1e-9 relative
    np.testing.assert_allclose(p.mean_velocity(f), u, rtol=2e-9)
    f = p.rest()
    p.run(f, 4000)
    np.testing.assert_allclose(p.mean_velocity(f), u, rtol=1e-8)


def test_tensor_z_invariant_reduces_to_the_2d_tensor_run():
    """A z-invariant K* with no coupling to z (K_xz = K_yz = K_zx = K_zy = 0) and no force along z
    evolves like the already pinned 2-D tensor run of its xy block (the exact D3Q19 -> D2Q9
    reduction, now through Eq. 18)."""
    K2 = _random_tensor_field((7, 8), seed=82)[..., :2, :2]
    K3 = np.zeros((3, 7, 8, 3, 3))
    K3[..., :2, :2] = K2[None]
    K3[..., 2, 2] = 5e-3
    tau, nu, eps, steps, g2 = 0.9, 0.08, 0.8, 150, (1.2e-6, -0.8e-6)
    p2 = oracle.Problem(tau, nu, eps, ktensor=K2.reshape(7, 8, 4), g=g2)
    f2 = p2.rest()
    p2.run(f2, steps)
    r2, u2, v2 = p2.fields(f2)
    p3 = oracle.Problem3D(tau, nu, eps, ktensor=K3, g=(g2[0], g2[1], 0.0))
    f3 = p3.rest()
    p3.run(f3, steps)
    r3, u3, v3, w3 = (t[1] for t in p3.fields(f3))
    scale = max(np.abs(u2).max(), np.abs(v2).max())
    np.testing.assert_allclose(r3, r2, rtol=0, atol=1e-14)
    np.testing.assert_allclose(u3, u2, rtol=0, atol=2e-9 * scale)
    np.testing.assert_allclose(v3, v2, rtol=0, atol=2e-9 * scale)
    assert np.abs(w3).max() <= 2e-9 * scale


def test_tensor_axis_permutation():
    """Relabelling the axes (x, y, z) -> (y, z, x) of the field, of K* (rows and columns) and of G
    permutes the velocity field the same way."""
    K = _random_tensor_field((4, 5, 6), seed=83)
    g = (1e-6, 2e-6, -1.5e-6)
    p = oracle.Problem3D(0.9, 0.1, 0.8, ktensor=K, g=g)
    f = p.rest()
    p.run(f, 80)
    r, u, v, w = p.fields(f)
    # new axes: x' = y, y' = z, z' = x; arrays [z'][y'][x'] = old [x][z][y]
    perm = [1, 2, 0]                                  # new component i is old component perm[i]
    Kp = np.transpose(K, (2, 0, 1, 3, 4))[..., perm, :][..., :, perm]
    q = oracle.Problem3D(0.9, 0.1, 0.8, ktensor=Kp, g=tuple(g[i] for i in perm))
    fq = q.rest()
    q.run(fq, 80)
    rq, uq, vq, wq = q.fields(fq)
    scale = max(np.abs(t).max() for t in (u, v, w))
    np.testing.assert_allclose(uq, np.transpose(v, (2, 0, 1)), rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(vq, np.transpose(w, (2, 0, 1)), rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(wq, np.transpose(u, (2, 0, 1)), rtol=0, atol=1e-9 * scale)


# ------------------------------------------------------- oversampled 3-D local problems

def test_oversampled_local3_periodic_embedding_is_exact():
    """A field that is periodic with the leaf's period: the cube grown by half a period on every
    side is two periods wide, its periodic solution is the leaf's solution repeated, and the
    inner-window mean equals the plain local problem's mean (up to summation order)."""
    s, m = 4, 2
    cube = synth.lognormal_kappa3d(s, s, s, 1.5, 1.5, seed=84).astype(np.float64)
    field = np.tile(cube, (3, 3, 3))
    grown = oracle.grown_cube(field, s, s, s, s, m)
    a = oracle.local_keff3(cube, 1.0, 1.0 / 6.0, 1.0, 1e-6, tol=0.0, max_steps=300)
    b = oracle.local_keff3(grown, 1.0, 1.0 / 6.0, 1.0, 1e-6, tol=0.0, max_steps=300, margin=m)
    np.testing.assert_allclose(b["keff"], a["keff"], rtol=0, atol=1e-12 * np.abs(a["keff"]).max())


def test_oversampled_local3_uniform_and_inner_layers():
    """A uniform grown cube gives kappa I. Parallel layers in the Darcy setting of Table 2
    (tau = 1/2, E3's nu and kappa ratio 10): bands of kappa_1 and kappa_2 across the inner leaf
    and margin bands of a third permeability. Drives along y and z see parallel layers, so
    K*_yy = K*_zz is the arithmetic mean over the columns averaged: the inner leaf's with
    oversampling, the whole cube's without."""
    s, m = 4, 2
    se = s + 2 * m
    r = oracle.local_keff3(np.full((se, se, se), 3e-3), 1.0, 1.0 / 6.0, 1.0, 1e-6, tol=1e-10, max_steps=100000,
                           margin=m)
    np.testing.assert_allclose(np.diag(r["keff"]), 3e-3, rtol=1e-6)
    ex = synth.paper_experiment("E3", ratio=10.0, ny=1)
    k1, k2 = float(ex["kappa"][0, 0]), float(ex["kappa"][0, 10])
    cols = np.array([5.0 * k2] * m + [k1] * 2 + [k2] * 2 + [5.0 * k2] * m)
    kap = np.broadcast_to(cols[None, None, :], (se, se, se)).copy()
    r = oracle.local_keff3(kap, ex["tau"], ex["nu"], ex["eps"], 1e-6, tol=1e-11, max_steps=20000, margin=m)
    inner = 0.5 * (k1 + k2)
    np.testing.assert_allclose([r["keff"][1, 1], r["keff"][2, 2]], inner, rtol=2e-6)
    full = oracle.local_keff3(kap, ex["tau"], ex["nu"], ex["eps"], 1e-6, tol=1e-11, max_steps=20000)
    np.testing.assert_allclose([full["keff"][1, 1], full["keff"][2, 2]], cols.mean(), rtol=2e-6)
    assert abs(full["keff"][1, 1] - inner) > 0.5 * inner


def test_tensor_layers_darcy_closed_form():
    """Layered full-tensor medium in the Darcy setting of Table 2 (tau = 1/2, E3's nu): K*(x)
    varies along x in bands of two cells, with non-symmetric K_xy, K_yx and K_zx; G along y.
    Steady Darcy flow u = K* (G - grad p) / nu with grad p = (p'(x), 0, 0): continuity makes u_x
    a constant c, periodicity makes p' average to zero, so c = G sum(K_xy / K_xx) /
    (nu sum(1 / K_xx)), p' = (K_xy G - nu c) / K_xx, u_y = (K_yy G - K_yx p') / nu and
    u_z = -K_zx p' / nu. A transposed or sign-flipped off-diagonal changes these at order one."""
    ex = synth.paper_experiment("E3", ratio=10.0, ny=1)
    k1 = float(ex["kappa"][0, 0])
    tau, nu, eps, g = ex["tau"], ex["nu"], ex["eps"], 1e-6
    band = lambda *v: np.repeat(np.array(v), 2) * k1          # noqa: E731
    kxx, kyy = band(2, 4, 1, 3), band(1, 5, 2, 8)
    kxy, kyx, kzx = band(0.3, -0.5, 0.2, 0.4), band(-0.2, 0.6, 0.1, -0.3), band(0.1, 0.2, -0.1, 0.3)
    nx = kxx.size
    K = np.zeros((3, 3, nx, 3, 3))
    K[..., 0, 0], K[..., 1, 1], K[..., 2, 2] = kxx, kyy, 3 * k1
    K[..., 0, 1], K[..., 1, 0], K[..., 2, 0] = kxy, kyx, kzx
    p = oracle.Problem3D(tau, nu, eps, ktensor=K, g=(0.0, g, 0.0))
    f = p.rest()
    p.run(f, 8000)
    _, u, v, w = p.fields(f)
    c = g * np.sum(kxy / kxx) / (nu * np.sum(1.0 / kxx))
    dp = (kxy * g - nu * c) / kxx
    np.testing.assert_allclose(u[1, 1, :], c, rtol=1e-5)
    np.testing.assert_allclose(v[1, 1, :], (kyy * g - kyx * dp) / nu, rtol=1e-5)
    uz = -kzx * dp / nu
    np.testing.assert_allclose(w[1, 1, :], uz, rtol=0, atol=1e-5 * np.abs(uz).max())
    for a in (u, v, w):                                    # uniform along y and z
        np.testing.assert_allclose(a, np.broadcast_to(a[1, 1, :], a.shape), rtol=0, atol=1e-12 * np.abs(v).max())
