"""Pins of the oracle's assembly, transfers, linear analysis, eigen-analysis and sensitivities.

Each test fixes the oracle to something other than itself: paper-printed DOF counts, exact Galerkin
identities of nested conforming spaces, dense linear algebra on tiny grids, the Euler closed form for
a slender column, the Rayleigh-quotient bound of eq. minBLFcharRayleigh, and central finite
differences of lambda_i and J with respect to single element densities.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

import synthetic
from oracle import assembly, grid, lba, sensitivity, transfer

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_dof_counts():
    cases = json.load(open(os.path.join(GOLDEN, "paper_counts.json")))["cases"]
    for c in cases:
        dim, nel = c["dim"], tuple(c["nel"]) + ((1,) if c["dim"] == 2 else ())
        n = dim * grid.num_nodes(nel, dim)
        if "dofs_rounded" in c:
            assert round(n / c["round_to"]) * c["round_to"] == pytest.approx(c["dofs_rounded"], rel=2e-3)
        if "elements" in c:
            assert int(np.prod(nel[:dim])) == c["elements"]
        if "coarsen" in c:
            lv = grid.level_nels(nel, dim, c["coarsen"] + 1)[-1]
            n = dim * grid.num_nodes(lv, dim)
        if "dofs" in c:
            assert n == c["dofs"]
        if "coarsen_ratio" in c:
            for k, ratio in c["coarsen_ratio"].items():
                lv = grid.level_nels(nel, dim, int(k) + 1)[-1]
                assert n / (dim * grid.num_nodes(lv, dim)) == pytest.approx(ratio, rel=0.02)


@pytest.mark.parametrize("dim", [2, 3])
def test_interpolation_partition_of_unity_and_linear_exactness(dim):
    nel = (4, 2, 2) if dim == 3 else (4, 2, 1)
    P = transfer.interpolation(nel, dim)
    assert np.allclose(P.sum(axis=1), 1.0)
    cn = grid.coarse_nel(nel, dim)
    def coords(ne):
        nd = grid.node_dims(ne, dim)
        if dim == 2:
            j, i = np.meshgrid(np.arange(nd[1]), np.arange(nd[0]), indexing="ij")
            return np.stack([i.reshape(-1), j.reshape(-1)], 1).astype(float)
        k, j, i = np.meshgrid(np.arange(nd[2]), np.arange(nd[1]), np.arange(nd[0]), indexing="ij")
        return np.stack([i.reshape(-1), j.reshape(-1), k.reshape(-1)], 1).astype(float)
    A = np.random.default_rng(0).standard_normal((dim, dim))
    uc = (2.0 * coords(cn) @ A.T).reshape(-1)      # coarse node at index I sits at fine coordinate 2I
    uf = (coords(nel) @ A.T).reshape(-1)
    assert np.allclose(P @ uc, uf)


@pytest.mark.parametrize("dim", [2, 3])
def test_galerkin_uniform_density_equals_coarse_stiffness(dim):
    """Nested conforming Q4/H8 spaces with exact quadrature: P^T K_h P = K_2h (unit elements on the
    coarse grid are twice as large; in 2D plane stress K scales as h^0, in 3D as h^1)."""
    nel = (4, 4, 2) if dim == 3 else (8, 4, 1)
    m = int(np.prod(nel[:dim]))
    Kh = assembly.assemble_K(nel, dim, np.ones(m), 0.3, 3.0, 1.0, 1e-6)
    P = transfer.interpolation(nel, dim)
    cn = grid.coarse_nel(nel, dim)
    K2h = assembly.assemble_K(cn, dim, np.ones(int(np.prod(cn[:dim]))), 0.3, 3.0, 1.0, 1e-6)
    scale = 1.0 if dim == 2 else 2.0
    assert np.allclose((P.T @ Kh @ P).toarray(), scale * K2h.toarray(), atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_galerkin_uniform_stress_equals_coarse_stress_stiffness(dim):
    """Under a linear displacement field (uniform stress) P^T G_h P = G_2h (same scaling as K)."""
    nel = (4, 4, 2) if dim == 3 else (8, 4, 1)
    cn = grid.coarse_nel(nel, dim)
    A = np.random.default_rng(3).standard_normal((dim, dim)) * 0.1
    def field(ne, h):
        nd = grid.node_dims(ne, dim)
        if dim == 2:
            j, i = np.meshgrid(np.arange(nd[1]), np.arange(nd[0]), indexing="ij")
            X = np.stack([i.reshape(-1), j.reshape(-1)], 1) * h
        else:
            k, j, i = np.meshgrid(np.arange(nd[2]), np.arange(nd[1]), np.arange(nd[0]), indexing="ij")
            X = np.stack([i.reshape(-1), j.reshape(-1), k.reshape(-1)], 1) * h
        return (X @ A.T).reshape(-1)
    m = int(np.prod(nel[:dim])); mc = int(np.prod(cn[:dim]))
    Gh = assembly.assemble_G(nel, dim, np.ones(m), field(nel, 1.0), 0.3, 3.0, 1.0, 1e-6)
    # coarse unit elements: the physical field at coarse node I (fine coordinate 2I), expressed
    # per coarse element of unit size, has gradient 2A; G scales with stress (x2) and 1/h^2 * h^d
    G2h = assembly.assemble_G(cn, dim, np.ones(mc), field(cn, 2.0), 0.3, 3.0, 1.0, 1e-6)
    P = transfer.interpolation(nel, dim)
    scale = 0.5 if dim == 2 else 1.0
    assert np.allclose((P.T @ Gh @ P).toarray(), scale * G2h.toarray(), atol=1e-12)


def test_global_K_symmetric_rigid_null_space():
    p = synthetic.column_2d(8, 4, seed=0, radius=2)
    K = assembly.assemble_K(p.nel, 2, p.x, p.nu, p.penal, p.E0, p.Emin)
    assert abs(K - K.T).max() < 1e-15
    n = p.num_dofs
    t = np.zeros(n); t[0::2] = 1.0
    assert np.abs(K @ t).max() < 1e-13


@pytest.mark.parametrize("shape", [(4, 2), (6, 2), (8, 4)])
def test_linear_analysis_direct_equals_dense(shape):
    p = synthetic.column_2d(*shape, seed=3, radius=1.5)
    op = lba.Problem(p)
    u, J = lba.linear_analysis(op)
    Kd = op.Kf.toarray()
    uf = np.linalg.solve(Kd, p.f[op.free])
    assert np.allclose(u[op.free], uf, rtol=1e-10, atol=1e-13 * np.abs(uf).max())
    assert J == pytest.approx(float(uf @ Kd @ uf), rel=1e-10)
    assert np.all(u[p.fixed == 1] == 0.0)


def test_linear_analysis_3d_direct_equals_dense():
    p = synthetic.cantilever_3d(2, 2, 2, seed=4, radius=1.5, volfrac=0.5)
    op = lba.Problem(p)
    u, J = lba.linear_analysis(op)
    uf = np.linalg.solve(op.Kf.toarray(), p.f[op.free])
    assert np.allclose(u[op.free], uf, rtol=1e-10)
    assert J == pytest.approx(float(p.f[op.free] @ uf), rel=1e-12)


def test_exact_lba_dense_brute_force_and_residual():
    p = synthetic.column_2d(12, 4, seed=5, radius=1.5)
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    lam, Phi, Gf = lba.exact_lba(op, u, 4)
    # brute force: all eigenvalues of the dense pencil K phi = lambda (-G) phi via K^{-1}(-G)
    Kd, Gd = op.Kf.toarray(), Gf.toarray()
    w = np.linalg.eigvals(np.linalg.solve(Kd, -Gd))
    w = np.real(w[np.abs(np.imag(w)) < 1e-12])
    brute = np.sort(1.0 / w[w > 1e-14])[:4]
    assert np.allclose(lam, brute, rtol=1e-9)
    for i in range(4):
        ph = Phi[op.free, i]
        assert ph @ Kd @ ph == pytest.approx(1.0, rel=1e-12)
        assert lba.eig_residual(op.Kf, Gf, lam[i], ph) < 1e-9
    assert np.abs(Phi[op.free].T @ Kd @ Phi[op.free] - np.eye(4)).max() < 1e-9


def test_sparse_lanczos_matches_dense_eigh():
    p = synthetic.column_2d(40, 16, seed=6, radius=2)
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    Gf = assembly.restrict_free(op.G(u), op.fixed)
    lam_d, Phi_d = lba.buckling_pencil(op.Kf, Gf, 6, dense_limit=10 ** 6)
    lam_s, Phi_s = lba.buckling_pencil(op.Kf, Gf, 6, dense_limit=10)
    assert np.allclose(lam_s, lam_d, rtol=1e-10)
    mac = np.abs(Phi_d.T @ op.Kf @ Phi_s)
    assert np.allclose(np.diag(mac), 1.0, atol=1e-7)


def test_euler_column_closed_form():
    """Uniform solid, slender clamped-free column of width w and length L = 40 w under a total
    compressive top load 1: lambda_1 -> pi^2 E (w^3/12) / (4 L^2) (plane stress, unit thickness).
    Q4 (bending locking) approaches it from above as the mesh is refined."""
    errs, ratios = [], []
    for across in (4, 8, 16):
        L = 40 * across
        p = synthetic.column_2d(L, across, seed=0, radius=1, x=np.ones(L * across))
        op = lba.Problem(p)
        u, _ = lba.linear_analysis(op)
        Gf = assembly.restrict_free(op.G(u), op.fixed)
        lam, _ = lba.buckling_pencil(op.Kf, Gf, 2, dense_limit=3000)
        exact = np.pi ** 2 * (across ** 3 / 12.0) / (4.0 * L ** 2)
        errs.append(lam[0] / exact - 1.0)
        ratios.append(lam[1] / lam[0])
    assert all(e > 0 for e in errs)
    assert errs[0] > 3.0 * errs[1] > 9.0 * errs[2]        # second-order convergence
    assert errs[2] < 0.005
    # second clamped-free Euler mode: (3 pi / 2)^2 / (pi / 2)^2 = 9
    assert ratios[2] == pytest.approx(9.0, rel=0.01)


def test_multilevel_rayleigh_bound_and_same_mesh_limit():
    p = synthetic.column_2d(24, 8, seed=7, radius=2)
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    lam, Phi, Gf = lba.exact_lba(op, u, 4)
    ml = lba.multilevel_lba(op, u, 4, eig_level=2)
    assert ml["lam"][0] >= lam[0] * (1 - 1e-12)
    assert np.all(ml["lam"] > 0)
    # eig_level = 1: coarse eigenpairs are the fine ones; one inverse-iteration step keeps them
    ml1 = lba.multilevel_lba(op, u, 4, eig_level=1)
    assert np.allclose(ml1["lam"], lam, rtol=1e-9)
    mac = np.abs(Phi[op.free].T @ op.Kf @ ml1["Phi"][op.free])
    assert np.allclose(np.diag(mac), 1.0, atol=1e-8)


def _fd_case():
    p = synthetic.column_2d(10, 4, seed=8, radius=1.5)
    return p


def _lba_values(p, q):
    op = lba.Problem(p)
    u, J = lba.linear_analysis(op)
    lam, Phi, Gf = lba.exact_lba(op, u, q)
    return op, u, J, lam, Phi


def test_sensitivities_central_difference():
    """Central FD with h = 1e-5 x_e on 20 random elements (exact LBA path), relative agreement
    1e-5 of max |dlambda_i/dx| where neighbouring eigenvalues are separated."""
    p = _fd_case()
    q = 3
    op, u, J, lam, Phi = _lba_values(p, q)
    dlam, dJ, Z = sensitivity.sensitivities(op, u, lam, Phi)
    gaps = np.minimum(np.abs(np.diff(np.r_[-np.inf, lam])), np.abs(np.diff(np.r_[lam, np.inf])))
    rng = np.random.default_rng(9)
    els = rng.choice(p.x.size, size=20, replace=False)
    x0 = p.x.copy()
    for e in els:
        h = 1e-5 * x0[e]
        vals = []
        for s in (+1, -1):
            p.x = x0.copy(); p.x[e] += s * h
            _, _, Js, lams, _ = _lba_values(p, q)
            vals.append((Js, lams))
        p.x = x0
        fdJ = (vals[0][0] - vals[1][0]) / (2 * h)
        assert fdJ == pytest.approx(dJ[e], abs=1e-5 * np.abs(dJ).max())
        fdl = (vals[0][1] - vals[1][1]) / (2 * h)
        for i in range(q):
            if gaps[i] / lam[i] > 1e-4:
                assert fdl[i] == pytest.approx(dlam[i, e], abs=1e-5 * np.abs(dlam[i]).max())


def test_adjoint_rhs_matches_directional_derivative_of_G():
    """b_k = phi^T (dG/du_k) phi: check b . w against (phi^T G[u + t w] phi - phi^T G[u - t w] phi)/2t."""
    p = synthetic.column_2d(6, 4, seed=10, radius=1.5)
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    rng = np.random.default_rng(11)
    phi = rng.standard_normal(p.num_dofs)
    w = rng.standard_normal(p.num_dofs)
    b = sensitivity.adjoint_rhs(p.nel, 2, p.x, phi, p.nu, p.penal, p.E0, p.Emin)
    t = 1e-3
    gp = phi @ (op.G(u + t * w) @ phi)
    gm = phi @ (op.G(u - t * w) @ phi)
    assert b @ w == pytest.approx((gp - gm) / (2 * t), rel=1e-10)


def test_batch_configs_shapes_and_levels():
    """The uneven 2D batch workload: 64 designs, 64 x 32 up to 512 x 256, aspect 2:1 to 4:1, each
    axis divisible by 2^(levels - 1), coarsest short side at most 8 elements."""
    import synthetic
    bs = synthetic.batch_configs()
    assert len(bs) == 64
    for p in bs:
        nx, ny = p.nel[0], p.nel[1]
        assert 32 <= nx <= 256 and ny in (2 * nx, 3 * nx, 4 * nx) and ny <= 512
        assert nx % 2 ** (p.mg_levels - 1) == 0 and ny % 2 ** (p.mg_levels - 1) == 0
        assert nx >> (p.mg_levels - 1) <= 8 or (nx >> (p.mg_levels - 1)) % 2 == 1
        assert 0.3 <= p.meta["volfrac"] <= 0.6 and abs(p.x.mean() - p.meta["volfrac"]) < 1e-5


def test_elementwise_apply_equals_assembled_operators():
    """The assembly-free K v and G v of the oracle (used for full-size checks) equal the assembled
    sparse operators."""
    import synthetic
    from oracle import assembly
    for p in (synthetic.column_2d(12, 6, seed=4, radius=2, mg_levels=1),
              synthetic.cantilever_3d(6, 4, 2, seed=5, radius=1.5, volfrac=0.4, mg_levels=1)):
        rng = np.random.default_rng(1)
        V = rng.standard_normal((2, p.num_dofs))
        u = rng.standard_normal(p.num_dofs)
        K = assembly.assemble_K(p.nel, p.dim, p.x, p.nu, p.penal, p.E0, p.Emin)
        G = assembly.assemble_G(p.nel, p.dim, p.x, u, p.nu, p.penal, p.E0, p.Emin)
        yk = assembly.apply_K(p.nel, p.dim, p.x, p.nu, p.penal, p.E0, p.Emin, V)
        yg = assembly.apply_G(p.nel, p.dim, p.x, u, p.nu, p.penal, p.E0, p.Emin, V)
        assert np.allclose(yk, (K @ V.T).T, rtol=1e-12, atol=1e-12 * np.abs(yk).max())
        assert np.allclose(yg, (G @ V.T).T, rtol=1e-12, atol=1e-12 * np.abs(yg).max())


# ------------------------------------------------------------------------------------------------
# multilevel chain (Sec. 2.1 steps 1-4) pinned by an independent coarse-mesh analysis
# ------------------------------------------------------------------------------------------------
def _roller_column(nel, dim, load, x0=0.8, mg_levels=3, eig_level=2, q=4):
    """Uniform column, long axis last (y in 2D, z in 3D): the base nodes ride on rollers (normal DOF
    fixed), one base corner is pinned in-plane (and in 3D a second base corner in y, which removes
    the rotation about z).  A compressive load of total magnitude `load` acts on the top as
    consistent nodal loads.  The exact solution is linear (uniform uniaxial stress, free Poisson
    expansion), so it lies in every coarse space of the hierarchy."""
    nd = [v + 1 for v in nel[:dim]]
    nn = int(np.prod(nd))
    n = dim * nn
    ids = np.arange(nn).reshape(nd[::-1])          # [z][y][x] or [y][x]
    fixed = np.zeros(n, dtype=np.uint8)
    f = np.zeros(n)
    if dim == 2:
        base, top = ids[0, :], ids[-1, :]
        w = np.full(nd[0], 1.0 / nel[0]); w[0] *= 0.5; w[-1] *= 0.5
        fixed[2 * base + 1] = 1
        fixed[2 * ids[0, 0]] = 1
        f[2 * top + 1] = -load * w
    else:
        base, top = ids[0].reshape(-1), ids[-1].reshape(-1)
        wx = np.ones(nd[0]); wx[0] = wx[-1] = 0.5
        wy = np.ones(nd[1]); wy[0] = wy[-1] = 0.5
        w = np.outer(wy, wx).reshape(-1) / float(nel[0] * nel[1])
        fixed[3 * base + 2] = 1
        fixed[3 * ids[0, 0, 0]] = fixed[3 * ids[0, 0, 0] + 1] = 1
        fixed[3 * ids[0, 0, -1] + 1] = 1
        f[3 * top + 2] = -load * w
    m = int(np.prod(nel[:dim]))
    nel3 = tuple(nel[:dim]) + ((1,) if dim == 2 else ())
    return synthetic.Problem(name="roller_column", dim=dim, nel=nel3, x=np.full(m, x0), f=f, fixed=fixed,
                             mg_levels=mg_levels, eig_level=eig_level, num_modes=q)


CHAIN_CASES = [(2, (8, 24), 2), (2, (8, 32), 3), (3, (4, 4, 8), 2)]


@pytest.mark.parametrize("dim,nel,level", CHAIN_CASES)
def test_multilevel_coarse_pencil_is_the_rediscretised_coarse_problem(dim, nel, level):
    """Uniform density and uniform stress: the Galerkin pencil (K^l, G^l) that multilevel_lba builds
    is the pencil of the same column re-meshed with elements 2^(l-1) times larger (Sec. 2.1 step 1;
    nested conforming spaces, exact quadrature).  On unit elements the coarse column is 2^(l-1)
    times smaller, so the load that keeps the stress is scaled by 2^-(l-1)(d-1); K and G then agree up
    to the common factor 2^(l-1)(d-2), which leaves the load factors unchanged.  The coarse load
    factors of multilevel_lba must equal those of an independent exact LBA of that coarse column."""
    q = 4
    p = _roller_column(nel, dim, 1.0, eig_level=level, mg_levels=level)
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    ml = lba.multilevel_lba(op, u, q, level)
    s = 2 ** (level - 1)
    pc = _roller_column(tuple(v // s for v in nel), dim, 1.0 / s ** (dim - 1), mg_levels=1, eig_level=1)
    opc = lba.Problem(pc)
    uc, _ = lba.linear_analysis(opc)
    lam_c, Phi_c, Gfc = lba.exact_lba(opc, uc, q)
    scale = float(s) ** (dim - 2)
    assert np.allclose(ml["Kl"].toarray(), scale * opc.Kf.toarray(), rtol=0, atol=1e-12 * abs(opc.Kf).max())
    assert np.allclose(ml["Gl"].toarray(), scale * Gfc.toarray(), rtol=0, atol=1e-12 * abs(Gfc).max())
    assert np.allclose(ml["lam_coarse"], lam_c, rtol=1e-10, atol=0), (ml["lam_coarse"], lam_c)


@pytest.mark.parametrize("dim,nel,level", CHAIN_CASES)
def test_multilevel_prolongated_modes_interpolate_the_coarse_modes(dim, nel, level):
    """Sec. 2.1 step 2 (Psi^j = I^j_{j+1} Psi^{j+1} down to Omega_1): at fine nodes that coincide
    with nodes of Omega_l the prolongated modes take the coarse nodal values; at the midpoint of two
    coinciding nodes along an axis they take their mean (bilinear / trilinear interpolation)."""
    q = 3
    p = _roller_column(nel, dim, 1.0, eig_level=level, mg_levels=level)
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    ml = lba.multilevel_lba(op, u, q, level)
    s = 2 ** (level - 1)
    ndf = [v + 1 for v in nel[:dim]]
    ndc = [v // s + 1 for v in nel[:dim]]
    fixed_c = ml["fixed_levels"][-1]
    Pc = np.zeros((dim * int(np.prod(ndc)), q))
    Pc[fixed_c == 0] = ml["Psi_coarse"]
    Pf = ml["Psi"].reshape(ndf[::-1] + [dim, q])
    Pc = Pc.reshape(ndc[::-1] + [dim, q])
    sl = tuple(slice(None, None, s) for _ in range(dim))
    assert np.allclose(Pf[sl], Pc, rtol=0, atol=1e-13 * np.abs(Pc).max())
    # midpoints along the first axis (x): mean of the two coarse neighbours
    if s >= 2:
        mid = tuple([slice(None, None, s)] * (dim - 1) + [slice(s // 2, None, s)])
        avg = 0.5 * (Pc[tuple([slice(None)] * (dim - 1) + [slice(0, -1)])]
                     + Pc[tuple([slice(None)] * (dim - 1) + [slice(1, None)])])
        assert np.allclose(Pf[mid], avg, rtol=0, atol=1e-13 * np.abs(Pc).max())


@pytest.mark.parametrize("dim,nel,level", CHAIN_CASES)
def test_multilevel_fine_step_brackets_the_load_factor(dim, nel, level):
    """Sec. 2.1 steps 3-4 are one inverse-iteration step of K^{-1}(-G) from the prolongated modes.
    Under pure compression -G is positive semi-definite, so the operator is positive semi-definite in
    the K inner product and one step cannot lower its Rayleigh quotient mu = 1/lambda: the fine load
    factor lies between the exact one (Rayleigh bound) and the coarse one (which is the fine Rayleigh
    quotient of the prolongated mode, by the Galerkin construction)."""
    q = 3
    p = _roller_column(nel, dim, 1.0, eig_level=level, mg_levels=level)
    op = lba.Problem(p)
    u, _ = lba.linear_analysis(op)
    Gf = lba.assembly.restrict_free(op.G(u), op.fixed)
    assert np.linalg.eigvalsh(-Gf.toarray()).min() > -1e-12 * abs(Gf).max()   # -G is PSD here
    ml = lba.multilevel_lba(op, u, q, level)
    lam_exact, _, _ = lba.exact_lba(op, u, 1)
    psi = ml["Psi"][op.free, 0]
    rq_psi = -(psi @ (op.Kf @ psi)) / (psi @ (Gf @ psi))
    assert rq_psi == pytest.approx(ml["lam_coarse"][0], rel=1e-10)
    assert lam_exact[0] * (1 - 1e-10) <= ml["lam"][0] <= ml["lam_coarse"][0] * (1 + 1e-10)
    # and the step really moves it (the coarse mode is not a fine eigenvector)
    assert ml["lam"][0] < ml["lam_coarse"][0] * (1 - 1e-6)
