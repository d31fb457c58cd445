"""GPU parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Inputs come from the seeded generators; expected values from ``oracle/`` only.  Floating
point tolerances: FP64 grids 1e-10 class, FP32 grids the stated targets (compliance 1e-5
relative, sensitivities 1e-4 guarded max-relative, products ~1e-6 relative).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem, filt, oc, topopt  # noqa: E402
from paper_2104_12282_gb300 import problems as P  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2104_12282_gb300 import tomo  # noqa: E402

DEV = torch.device("cuda:0")


def f32(a):
    """Round to float32 and back: both sides then see identical inputs."""
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


def T(a, prec):
    dt = torch.float64 if prec == tomo.FP64 else torch.float32
    return torch.tensor(np.asarray(a), dtype=dt, device=DEV)


def H(t):
    return t.detach().cpu().numpy().astype(np.float64)


def guarded_rel(x, ref):
    """max |x - ref| / max(|ref|, 1e-3 max|ref|), elementwise, then max."""
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return float(np.max(np.abs(x - ref) / den))


SMALL = [(1, 1, 1), (2, 1, 1), (3, 2, 5), (17, 9, 5), (33, 17, 9), (45, 21, 13), (7, 31, 4)]


def _problem(kind, dims):
    if kind == "cantilever":
        return P.cantilever(*dims)
    return P.mbb_block(*dims, rmin=1.5)


# ---------------------------------------------------------------------------------------
# S3: matrix-free product
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [tomo.FP64, tomo.FP32])
@pytest.mark.parametrize("dims", SMALL)
@pytest.mark.parametrize("kind", ["cantilever", "mbb"])
def test_apply_stiffness_matches_oracle(prec, dims, kind):
    p = _problem(kind, dims)
    d = p.dims
    rho = f32(P.random_field(d, 1, 0.05, 1.0))
    x = f32(P.random_nodal(d, 2))
    m = topopt.Model(p)
    E = m.modulus(rho)
    K = fem.assemble(d.nx, d.ny, d.nz, E, p.h, m.K0)
    free = ~m.fixed
    ref = np.where(free, K @ np.where(free, x, 0.0), 0.0)
    with tomo.Grid.from_problem(p, precision=prec) as g:
        y = torch.empty(d.n_dof, dtype=T([0.0], prec).dtype, device=DEV)
        g.apply_stiffness(T(rho, prec), T(x, prec), y)
        torch.cuda.synchronize()
        got = H(y)
    scale = np.abs(ref).max()
    tol = 1e-13 if prec == tomo.FP64 else 2e-6
    assert np.abs(got - ref).max() <= tol * scale, np.abs(got - ref).max() / scale
    assert np.all(got[~free] == 0.0)


@pytest.mark.parametrize("prec", [tomo.FP64, tomo.FP32])
def test_apply_stiffness_smooth_field_accuracy(prec):
    """On a smooth displacement (a near-rigid field plus small strains) the FP32 product
    keeps its rounding relative to the strains (differences-first transform)."""
    p = P.cantilever(40, 20, 20)
    d = p.dims
    nn = d.n_nodes
    k, j, i = np.meshgrid(np.arange(d.nz + 1), np.arange(d.ny + 1), np.arange(d.nx + 1),
                          indexing="ij")
    X = np.stack([i.ravel(), j.ravel(), k.ravel()], 1).astype(float)
    u = np.zeros(3 * nn)
    u[:nn] = 100.0 + 1e-3 * np.sin(X[:, 0] / 7.0) * X[:, 1]
    u[nn:2 * nn] = -50.0 + 1e-3 * np.cos(X[:, 2] / 5.0)
    u[2 * nn:] = 75.0 + 1e-3 * X[:, 0] * X[:, 2] / 40.0
    u = f32(u)
    rho = f32(P.random_field(d, 3, 0.3, 1.0))
    m = topopt.Model(p)
    E = m.modulus(rho)
    ref = m.apply(E, u)
    with tomo.Grid.from_problem(p, precision=prec) as g:
        y = torch.empty(d.n_dof, dtype=T([0.0], prec).dtype, device=DEV)
        g.apply_stiffness(T(rho, prec), T(u, prec), y)
        torch.cuda.synchronize()
        got = H(y)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= (1e-12 if prec == tomo.FP64 else 1e-4), err


# ---------------------------------------------------------------------------------------
# S1/S7: filter
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [tomo.FP64, tomo.FP32])
@pytest.mark.parametrize("rmin", [1.0, 1.5, 2.5, 3.3, 5.5, 7.2])
@pytest.mark.parametrize("dims", [(1, 1, 1), (17, 9, 5), (40, 13, 11)])
def test_filter_matches_oracle(prec, rmin, dims):
    p = P.cantilever(*dims, rmin=rmin)
    d = p.dims
    z = f32(P.random_field(d, 4, 0.0, 1.0))
    x = f32(P.random_sensitivity(d, 5))
    fwd = filt.filter_forward(d.nx, d.ny, d.nz, rmin, z)
    tr = filt.filter_transpose(d.nx, d.ny, d.nz, rmin, x)
    # Summation bound: n terms summed in any order carry at most (n - 1) u sum|terms|, plus
    # the division by Hs; elementwise against the same filter of |input|.
    u = 2.0 ** -53 if prec == tomo.FP64 else 2.0 ** -24
    bound = (len(filt.stencil_offsets(rmin)) + 2) * u
    scale_f = filt.filter_forward(d.nx, d.ny, d.nz, rmin, np.abs(z))
    scale_t = filt.filter_transpose(d.nx, d.ny, d.nz, rmin, np.abs(x))
    with tomo.Grid.from_problem(p, precision=prec) as g:
        out = T(np.zeros(d.n_el), prec)
        g.filter(T(z, prec), out)
        torch.cuda.synchronize()
        assert np.all(np.abs(H(out) - fwd) <= bound * scale_f + 1e-300)
        g.filter(T(x, prec), out, transpose=True)
        torch.cuda.synchronize()
        assert np.all(np.abs(H(out) - tr) <= bound * scale_t + 1e-300)


# ---------------------------------------------------------------------------------------
# S3-S5: state solve
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("kind,dims", [("cantilever", (24, 12, 12)), ("mbb", (33, 17, 9)),
                                       ("cantilever", (5, 3, 2))])
def test_solve_fp64_matches_direct(kind, dims):
    p = _problem(kind, dims)
    d = p.dims
    rho = f32(P.random_field(d, 6, 0.05, 1.0))
    m = topopt.Model(p)
    uref, _, _ = m.solve(m.modulus(rho), "direct")
    with tomo.Grid.from_problem(p, precision=tomo.FP64, rtol=1e-12, maxit=5000) as g:
        u = T(np.zeros(d.n_dof), tomo.FP64)
        info = g.solve(T(rho, tomo.FP64), u)
        torch.cuda.synchronize()
    assert info.status == 0 and info.rel_res <= 1e-12
    assert np.abs(H(u) - uref).max() <= 1e-9 * np.abs(uref).max()


@pytest.mark.parametrize("precond", [tomo.PRECOND_MG, tomo.PRECOND_JACOBI])
def test_solve_fp32_matches_direct(precond):
    p = P.cantilever(24, 12, 12)
    d = p.dims
    rho = f32(P.random_field(d, 7, 0.05, 1.0))
    m = topopt.Model(p)
    uref, _, _ = m.solve(m.modulus(rho), "direct")
    cref = p.f @ uref
    with tomo.Grid.from_problem(p, precision=tomo.FP32, rtol=1e-6, precond=precond) as g:
        u = T(np.zeros(d.n_dof), tomo.FP32)
        info = g.solve(T(rho, tomo.FP32), u)
        torch.cuda.synchronize()
    assert info.status == 0 and info.rel_res <= 1e-6
    c = p.f @ H(u)
    assert abs(c / cref - 1.0) <= 1e-5, abs(c / cref - 1.0)


def test_multigrid_beats_jacobi_iterations():
    p = P.cantilever(48, 24, 24)
    rho = f32(P.random_field(p.dims, 8, 0.05, 1.0))
    its = {}
    for pc in (tomo.PRECOND_MG, tomo.PRECOND_JACOBI):
        with tomo.Grid.from_problem(p, precision=tomo.FP32, precond=pc, maxit=5000) as g:
            u = T(np.zeros(p.dims.n_dof), tomo.FP32)
            its[pc] = g.solve(T(rho, tomo.FP32), u).iters
    assert its[tomo.PRECOND_MG] * 5 < its[tomo.PRECOND_JACOBI], its


@pytest.mark.parametrize("kind", ["cantilever", "mbb"])
def test_residual_of_float_pair_matches_oracle(kind):
    """r = f - K (u_hi + u_lo) with the pair input: at the oracle's solution the FP32 kernel
    returns a residual at FP32 rounding level, far below that of u_hi alone."""
    p = _problem(kind, (33, 17, 9))
    d = p.dims
    rho = f32(P.random_field(d, 17, 0.05, 1.0))
    m = topopt.Model(p)
    E = m.modulus(rho)
    u, _, _ = m.solve(E, "direct")
    uhi = u.astype(np.float32)
    ulo = (u - uhi.astype(np.float64)).astype(np.float32)
    ref_hi = np.where(m.fixed, 0.0, p.f - m.apply(E, uhi.astype(np.float64)))
    # size of the terms the product sums: || |K| |u| ||
    scale = np.linalg.norm(np.where(m.fixed, 0.0, fem.apply_elementwise(
        d.nx, d.ny, d.nz, E, p.h, np.abs(m.K0), np.abs(uhi.astype(np.float64)))))
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        r = torch.empty(d.n_dof, dtype=torch.float32, device=DEV)
        g.residual(T(rho, tomo.FP32), T(uhi, tomo.FP32), r, u_lo=T(ulo, tomo.FP32))
        torch.cuda.synchronize()
        r_pair = H(r)
        g.residual(T(rho, tomo.FP32), T(uhi, tomo.FP32), r)
        torch.cuda.synchronize()
        r_hi = H(r)
    # residual of u_hi alone: the oracle's FP64 residual of u_hi up to the FP32 rounding of
    # the product, which the differences-first transform keeps far below eps * |K||u|
    assert np.linalg.norm(r_hi - ref_hi) <= 1e-9 * scale
    # pair: the exact solution's residual is 0, so only that rounding remains, well below
    # the residual caused by rounding u itself to float
    assert np.linalg.norm(r_pair) <= 1e-9 * scale
    assert np.linalg.norm(r_pair) <= 0.2 * np.linalg.norm(ref_hi)


@pytest.mark.parametrize("prec", [tomo.FP64, tomo.FP32])
def test_residual_replacement_keeps_convergence(prec):
    """Jacobi-PCG with the residual replaced (in FP64) every 10 iterations converges like
    the plain recurrence and to the same compliance."""
    p = P.cantilever(24, 12, 12)
    rho = f32(P.random_field(p.dims, 18, 0.05, 1.0))
    m = topopt.Model(p)
    cref = p.f @ m.solve(m.modulus(rho), "direct")[0]
    its = {}
    for rr in (-1, 10):
        with tomo.Grid.from_problem(p, precision=prec, precond=tomo.PRECOND_JACOBI,
                                    maxit=5000, rr_every=rr) as g:
            u = T(np.zeros(p.dims.n_dof), prec)
            info = g.solve(T(rho, prec), u)
            torch.cuda.synchronize()
            its[rr] = info.iters
            assert abs(p.f @ H(u) / cref - 1.0) <= 1e-5
    assert its[10] <= 1.2 * its[-1] + 5, its


# ---------------------------------------------------------------------------------------
# S6: sensitivity (same u on both sides, from the oracle)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [tomo.FP64, tomo.FP32])
@pytest.mark.parametrize("dims", [(3, 2, 5), (33, 17, 9)])
def test_sensitivity_matches_oracle(prec, dims):
    p = P.cantilever(*dims)
    d = p.dims
    rho = f32(P.random_field(d, 9, 0.05, 1.0))
    m = topopt.Model(p)
    u, _, _ = m.solve(m.modulus(rho), "direct")
    u = f32(u)
    dref = m.sensitivity(rho, u)
    cref = p.f @ u
    with tomo.Grid.from_problem(p, precision=prec) as g:
        dc = T(np.zeros(d.n_el), prec)
        c = g.sensitivity(T(rho, prec), T(u, prec), dc)
        torch.cuda.synchronize()
    # FP64: the oracle's u_e^T K0 u_e is a plain 24x24 quadratic form, which cancels the
    # rigid-body part of u_e in FP64 and is itself only good to ~1e-10 where the strains are
    # small against the displacements; the GPU forms differences first.
    tol = 1e-9 if prec == tomo.FP64 else 1e-4
    assert guarded_rel(H(dc), dref) <= tol
    assert abs(c / cref - 1.0) <= (1e-13 if prec == tomo.FP64 else 1e-6)


# ---------------------------------------------------------------------------------------
# S1-S7: exact gradient
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [tomo.FP64, tomo.FP32])
@pytest.mark.parametrize("kind,dims,rmin", [("cantilever", (24, 12, 12), 1.5),
                                            ("mbb", (33, 17, 9), 2.5)])
def test_gradient_matches_oracle(prec, kind, dims, rmin):
    p = P.cantilever(*dims, rmin=rmin) if kind == "cantilever" else P.mbb_block(*dims, rmin=rmin)
    d = p.dims
    z = f32(P.bumpy_field(d, 10, sigma=(2.0, 6.0)))
    m = topopt.Model(p)
    ref = m.gradient(z, "direct")
    rtol = 1e-12 if prec == tomo.FP64 else 1e-6
    with tomo.Grid.from_problem(p, precision=prec, rtol=rtol, maxit=5000) as g:
        dcdz = T(np.zeros(d.n_el), prec)
        dvdz = T(np.zeros(d.n_el), prec)
        c, info = g.gradient(T(z, prec), dcdz, dvdz)
        torch.cuda.synchronize()
    if prec == tomo.FP64:
        assert abs(c / ref["c"] - 1.0) <= 1e-10
        assert guarded_rel(H(dcdz), ref["dcdz"]) <= 1e-9
        assert np.abs(H(dvdz) - ref["dvdz"]).max() <= 1e-14
    else:
        assert abs(c / ref["c"] - 1.0) <= 1e-5
        assert guarded_rel(H(dcdz), ref["dcdz"]) <= 1e-4
        assert np.abs(H(dvdz) - ref["dvdz"]).max() <= 1e-6


@pytest.mark.parametrize("prec", [tomo.FP64, tomo.FP32])
def test_device_loop_and_host_loop_agree(prec):
    """The conditional-graph CG loop and the host-issued loop (used while profiling) run the
    same kernels in the same order: results are bitwise equal."""
    p = P.mbb_block(33, 17, 9, rmin=2.5)
    z = f32(P.bumpy_field(p.dims, 16, sigma=(2.0, 6.0)))
    with tomo.Grid.from_problem(p, precision=prec, rr_every=3) as g:
        zt = T(z, prec)
        dc1 = torch.empty_like(zt)
        dc2 = torch.empty_like(zt)
        c1, i1 = g.gradient(zt, dc1)
        g.profile_enable(True)
        c2, i2 = g.gradient(zt, dc2)
        n, ms, b = g.profile_read()
        g.profile_enable(False)
        torch.cuda.synchronize()
    assert i1.iters == i2.iters and i1.iters > 3
    assert c1 == c2 and torch.equal(dc1, dc2)
    assert n > 0 and ms > 0 and b > 0
    if prec == tomo.FP32:
        # the fine-level products that did work: four in the first V-cycle (degree 2: one
        # Chebyshev step after the Jacobi start, the residual, two post-smoothing steps),
        # then per iteration the CG product, and for every iteration but the last (which
        # stops at its convergence test) another V-cycle's four: 5 per iteration
        assert n == 5 * i2.iters


def test_gradient_host_buffers_equal_device_buffers():
    p = P.cantilever(17, 9, 5)
    d = p.dims
    z = f32(P.random_field(d, 11, 0.1, 1.0)).astype(np.float32)
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        dc_h = np.zeros(d.n_el, np.float32)
        dv_h = np.zeros(d.n_el, np.float32)
        c_h, _ = g.gradient(z, dc_h, dv_h)
        zt = torch.tensor(z, device=DEV)
        dc_d = torch.empty_like(zt)
        dv_d = torch.empty_like(zt)
        c_d, _ = g.gradient(zt, dc_d, dv_d)
        torch.cuda.synchronize()
    assert c_h == c_d
    assert np.array_equal(dc_h, dc_d.cpu().numpy()) and np.array_equal(dv_h, dv_d.cpu().numpy())


# ---------------------------------------------------------------------------------------
# S8: OC update (oracle inputs on both sides)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [tomo.FP64, tomo.FP32])
@pytest.mark.parametrize("n,volfrac,move", [((20, 10, 10), 0.3, 0.2), ((33, 17, 9), 0.12, 0.2),
                                            ((8, 4, 4), 0.5, 1.0), ((1, 1, 1), 0.5, 0.2)])
def test_oc_step_matches_oracle(prec, n, volfrac, move):
    p = P.cantilever(*n, volfrac=volfrac)
    d = p.dims
    z = f32(P.random_field(d, 12, 0.0, 1.0))
    dc = f32(P.random_sensitivity(d, 13))
    dv = f32(filt.filter_transpose(d.nx, d.ny, d.nz, p.rmin, np.ones(d.n_el)))
    vmax = volfrac * d.n_el
    zr, lam, chr_ = oc.oc_update(z, dc, dv, vmax, move)
    with tomo.Grid.from_problem(p, precision=prec) as g:
        zn = T(np.zeros(d.n_el), prec)
        ch = g.oc_step(T(z, prec), T(dc, prec), T(dv, prec), volfrac, move, zn)
        torch.cuda.synchronize()
    tol = 1e-9 if prec == tomo.FP64 else 1e-5
    assert np.abs(H(zn) - zr).max() <= tol
    assert abs(ch - chr_) <= tol


def test_oc_step_infeasible_volume_goes_to_lower_bounds():
    p = P.cantilever(10, 5, 5)
    d = p.dims
    z = f32(P.random_field(d, 14, 0.5, 1.0))
    dc = f32(P.random_sensitivity(d, 15))
    dv = np.ones(d.n_el)
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        zn = T(np.zeros(d.n_el), tomo.FP32)
        g.oc_step(T(z, tomo.FP32), T(dc, tomo.FP32), T(dv, tomo.FP32), 0.05, 0.2, zn)
        torch.cuda.synchronize()
    assert np.abs(H(zn) - np.maximum(0.0, z - 0.2)).max() <= 1e-6


# ---------------------------------------------------------------------------------------
# Whole loop: the 24x12x12 cantilever, 10 OC iterations
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", [tomo.FP64, tomo.FP32])
def test_oc_trajectory_matches_oracle(prec):
    p = P.cantilever_24x12x12()
    d = p.dims
    m = topopt.Model(p)
    _, hist = m.run(p.meta["oc_iters"], method="direct")
    rtol = 1e-12 if prec == tomo.FP64 else 1e-6
    cs = []
    with tomo.Grid.from_problem(p, precision=prec, rtol=rtol, maxit=5000) as g:
        z = T(p.z0, prec)
        dc = torch.empty_like(z)
        dv = torch.empty_like(z)
        zn = torch.empty_like(z)
        for _ in range(p.meta["oc_iters"]):
            c, _ = g.gradient(z, dc, dv)
            g.oc_step(z, dc, dv, p.volfrac, p.move, zn)
            z, zn = zn, z
            cs.append(c)
    cref = np.array([h["c"] for h in hist])
    rel = np.abs(np.array(cs) / cref - 1.0)
    assert rel.max() <= (1e-8 if prec == tomo.FP64 else 1e-5), rel


# ---------------------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------------------
def test_zero_load_gives_zero_solution():
    p = P.cantilever(6, 3, 3)
    p.f[:] = 0.0
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        z = T(np.full(p.n_el, 0.5), tomo.FP32)
        dc = torch.empty_like(z)
        c, info = g.gradient(z, dc)
        torch.cuda.synchronize()
    assert c == 0.0 and info.iters == 0 and torch.all(dc == 0)


def test_wrong_precision_and_sizes_are_rejected():
    p = P.cantilever(6, 3, 3)
    with tomo.Grid.from_problem(p, precision=tomo.FP32) as g:
        with pytest.raises(TypeError):
            g.filter(torch.zeros(p.n_el, dtype=torch.float64, device=DEV),
                     torch.zeros(p.n_el, dtype=torch.float64, device=DEV))
        with pytest.raises(ValueError):
            g.filter(torch.zeros(p.n_el + 1, device=DEV), torch.zeros(p.n_el + 1, device=DEV))
        st = tomo.lib().tomo_filter_d(g._h, None, None, 0)
        assert st == 1
        assert b"precision" in tomo.lib().tomo_last_error(g._h)


def test_maxit_reports_no_convergence():
    p = P.cantilever(24, 12, 12)
    with tomo.Grid.from_problem(p, precision=tomo.FP32, maxit=2, rtol=1e-12) as g:
        z = T(np.full(p.n_el, 0.4), tomo.FP32)
        dc = torch.empty_like(z)
        with pytest.raises(tomo.TomoError) as e:
            g.gradient(z, dc)
    assert e.value.status == 3


@pytest.mark.parametrize("rr", [1, 3])
def test_multigrid_with_frequent_residual_replacement(rr):
    """FP32 multigrid-PCG whose FP64 residual replacement runs every rr iterations (it then
    also renews the finest level's first smoothing step): same solution as the oracle."""
    p = P.cantilever(24, 12, 12)
    rho = f32(P.random_field(p.dims, 19, 0.05, 1.0))
    m = topopt.Model(p)
    ref = m.gradient(rho, "direct")
    with tomo.Grid.from_problem(p, precision=tomo.FP32, rr_every=rr) as g:
        z = T(rho, tomo.FP32)
        dc = torch.empty_like(z)
        c, info = g.gradient(z, dc)
        torch.cuda.synchronize()
    assert info.status == 0 and info.iters > rr
    assert abs(c / ref["c"] - 1.0) <= 1e-5
    assert guarded_rel(H(dc), ref["dcdz"]) <= 1e-4
