"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
hand-derived worked examples (tests/golden), closed forms, invariances,
central finite differences, library routines (scipy rotations, dense solves)
and textbook properties of CG / GN / LM.  CPU only.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import energies as en
from oracle import solver as so
from paper_1604_06525_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def fd_jacobian(energy, x, h=1e-6):
    cols = []
    for i in range(x.size):
        e = np.zeros_like(x)
        e[i] = h
        cols.append((energy.residuals(x + e) - energy.residuals(x - e)) / (2 * h))
    return np.stack(cols, 1)


def tiny_warp(W=4, H=3, n_handles=2, seed=3, mask_frac=0.0, noise=0.3):
    mask = synth.random_mask(W, H, mask_frac, seed + 7) if mask_frac > 0 else None
    return synth.warp_problem(W, H, n_handles, seed=seed, mask=mask, x0_noise=noise)


def tiny_mesh(level=0, seed=5, noise=0.3):
    return synth.mesh_problem(level, seed=seed, handle_frac=0.2, x0_noise=noise)


# --------------------------------------------------------------------------
# worked examples derived by hand (tests/golden/*.json)
# --------------------------------------------------------------------------
def test_golden_warp_3x1():
    g = _golden("warp_3x1.json")
    prob = synth.warp_problem(g["W"], g["H"], 0, seed=0)
    prob.handle_idx = np.array(g["handle_idx"], np.int32)
    prob.handle_target = np.array(g["handle_target"], np.float32)
    prob.w_reg, prob.w_fit = g["w_reg"], g["w_fit"]
    e = en.WarpEnergy(prob)
    x = np.array(g["x"], np.float64).reshape(-1)
    jtf, diag, E = so.jtf_diag(e, x)
    assert E == pytest.approx(g["E"], abs=1e-12)
    np.testing.assert_allclose(jtf, np.array(g["jtf"]).reshape(-1), atol=1e-12)
    np.testing.assert_allclose(diag, np.array(g["diag"]).reshape(-1), atol=1e-12)


def test_golden_mesh_2v():
    g = _golden("mesh_2v.json")
    U = np.array(g["urshape"], np.float32)
    prob = synth.graph_problem(U, g["v0"], g["v1"], 0)
    e = en.MeshEnergy(prob)
    x = np.array(g["x"], np.float64).reshape(-1)
    jtf, diag, E = so.jtf_diag(e, x)
    assert E == pytest.approx(g["E"], abs=1e-12)
    np.testing.assert_allclose(jtf, np.array(g["jtf"]).reshape(-1), atol=1e-12)
    np.testing.assert_allclose(diag, np.array(g["diag"]).reshape(-1), atol=1e-12)


def test_golden_poisson_3x1():
    g = _golden("poisson_3x1.json")
    W, H = g["W"], g["H"]
    prob = synth.PoissonProblem(W, H, np.array(g["X"], np.float32).reshape(4, H, W),
                                np.array(g["T"], np.float32).reshape(4, H, W),
                                np.array(g["mask"], np.uint8).reshape(H, W))
    e = en.PoissonEnergy(prob)
    jtf, diag, E = so.jtf_diag(e, prob.x0.reshape(-1))
    assert E == pytest.approx(g["E"], abs=1e-12)
    np.testing.assert_allclose(jtf[:W * H], g["jtf_c0"], atol=1e-12)
    np.testing.assert_allclose(diag[:W * H], g["diag_c0"], atol=1e-12)
    # the other channels see the same structure (diag) and zero data
    np.testing.assert_allclose(diag[W * H:2 * W * H], g["diag_c0"], atol=1e-12)
    np.testing.assert_allclose(jtf[W * H:], 0.0, atol=1e-12)


# --------------------------------------------------------------------------
# residuals / energy: closed forms and invariances
# --------------------------------------------------------------------------
def test_warp_rest_state_is_zero():
    prob = synth.warp_problem(9, 7, 5, seed=1, max_disp=0.0)
    e = en.WarpEnergy(prob)
    jtf, _, E = so.jtf_diag(e, prob.x0.reshape(-1))
    assert E == 0.0
    assert np.abs(jtf).max() == 0.0


def test_warp_fit_closed_form_weight_convention():
    # at the rest state every regularizer residual vanishes, so
    # E = w_fit * sum |target|^2  (the weight multiplies the squared residual)
    prob = synth.warp_problem(11, 6, 9, seed=2)
    E = en.WarpEnergy(prob).energy(prob.x0.reshape(-1))
    t = prob.handle_target.astype(np.float64)
    assert E == pytest.approx(prob.w_fit * float((t * t).sum()), rel=1e-13)


@pytest.mark.parametrize("mask_frac", [0.0, 0.3])
def test_warp_scaling_counts_valid_residuals(mask_frac):
    # O = 2 U (displacement = U), theta = 0: every residual equals U_k - U_{k+d}
    # (unit length on the lattice), so E_reg = w_reg * #valid directed pairs.
    W, H = 7, 5
    mask = synth.random_mask(W, H, mask_frac, 11) if mask_frac else None
    prob = synth.warp_problem(W, H, 0, seed=4, mask=mask)
    prob.w_reg = 2.5
    x = np.concatenate([prob.urshape.reshape(-1), np.zeros(W * H)])
    count = 0
    for y in range(H):
        for xx in range(W):
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                nx, ny = xx + dx, y + dy
                if not (0 <= nx < W and 0 <= ny < H):
                    continue
                if mask is not None and (mask[y, xx] or mask[ny, nx]):
                    continue
                count += 1
    assert en.WarpEnergy(prob).energy(x) == pytest.approx(2.5 * count, rel=1e-13)


def test_warp_rigid_motion_has_zero_regularizer():
    # O = Rot(phi) U + t with theta = phi everywhere: rigid, so E_reg = 0.
    # The rotation comes from scipy (counter-clockwise about z), not the oracle.
    W, H = 8, 6
    prob = synth.warp_problem(W, H, 0, seed=5)
    phi = 0.7
    Rm = Rotation.from_euler("z", phi).as_matrix()[:2, :2]
    U = prob.urshape.reshape(2, -1).astype(np.float64)
    O = Rm @ U + np.array([[3.0], [-2.0]])
    x = np.concatenate([(O - U).reshape(-1), np.full(W * H, phi)])
    assert en.WarpEnergy(prob).energy(x) < 1e-20
    # a clockwise rotation of the same angle is not rigid for theta = phi
    x_bad = np.concatenate([(Rm.T @ U - U).reshape(-1), np.full(W * H, phi)])
    assert en.WarpEnergy(prob).energy(x_bad) > 1.0


def test_poisson_guidance_copy_is_zero_energy():
    # X = T + const: every gradient matches the guidance, E = 0
    prob = synth.poisson_problem(20, 14, seed=6)
    x = prob.guide.astype(np.float64) + 0.25
    assert en.PoissonEnergy(prob).energy(x.reshape(-1)) < 1e-24


def test_euler_convention_matches_scipy_extrinsic_xyz():
    rng = np.random.default_rng(0)
    A = rng.uniform(-2, 2, size=(16, 3))
    R, dR = en.euler_rotation(A)
    ref = Rotation.from_euler("xyz", A).as_matrix()   # extrinsic x, y, z = Rz Ry Rx
    np.testing.assert_allclose(R, ref, atol=1e-14)
    h = 1e-6
    for m in range(3):
        e = np.zeros(3)
        e[m] = h
        fd = (Rotation.from_euler("xyz", A + e).as_matrix()
              - Rotation.from_euler("xyz", A - e).as_matrix()) / (2 * h)
        np.testing.assert_allclose(dR[m], fd, atol=1e-8)


def test_mesh_rest_state_is_zero_and_fit_closed_form():
    prob = synth.mesh_problem(1, seed=3)
    e = en.MeshEnergy(prob)
    t = prob.handle_target.astype(np.float64)
    assert e.energy(prob.x0.reshape(-1)) == pytest.approx(prob.w_fit * float((t * t).sum()), rel=1e-13)
    prob.handle_target[:] = 0
    jtf, _, E = so.jtf_diag(en.MeshEnergy(prob), prob.x0.reshape(-1))
    assert E == 0.0 and np.abs(jtf).max() == 0.0


def test_mesh_rigid_motion_and_scaling():
    prob = synth.mesh_problem(2, seed=4)
    prob.handle_idx = prob.handle_idx[:0]
    prob.handle_target = prob.handle_target[:0]
    e = en.MeshEnergy(prob)
    U = prob.urshape.astype(np.float64)
    ang = np.array([0.3, -1.1, 2.0])
    Rm = Rotation.from_euler("xyz", ang).as_matrix()
    O = Rm @ U + np.array([[0.5], [1.0], [-2.0]])
    x = np.concatenate([(O - U).reshape(-1), np.repeat(ang, prob.V)])
    assert e.energy(x) < 1e-20
    # scaling O = 2U: E_reg = w_reg * sum over directed edges |U_a - U_b|^2
    x2 = np.concatenate([U.reshape(-1), np.zeros(3 * prob.V)])
    dU = U[:, prob.v0] - U[:, prob.v1]
    assert e.energy(x2) == pytest.approx(float((dU * dU).sum()), rel=1e-12)


def test_mesh_on_grid_graph_reduces_to_image_warp():
    # A planar grid given as an explicit graph with rotations about z only is
    # the image-warping energy (Sec. 8.4 compares exactly these two forms).
    W, H = 5, 4
    wp = synth.warp_problem(W, H, 3, seed=8, x0_noise=0.4)
    ys, xs = np.mgrid[0:H, 0:W]
    v0, v1 = [], []
    for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        nx, ny = xs + dx, ys + dy
        ok = (nx >= 0) & (nx < W) & (ny >= 0) & (ny < H)
        v0.append((ys * W + xs)[ok])
        v1.append((ny * W + nx)[ok])
    U3 = np.concatenate([wp.urshape.reshape(2, -1), np.zeros((1, W * H), np.float32)])
    mp = synth.graph_problem(U3, np.concatenate(v0), np.concatenate(v1), 0)
    mp.handle_idx = wp.handle_idx
    mp.handle_target = np.concatenate([wp.handle_target, np.zeros((3, 1), np.float32)], 1)
    xw = wp.x0.reshape(3, -1).astype(np.float64)
    xm = np.concatenate([xw[0:2], np.zeros((3, W * H)), xw[2:3]]).reshape(-1)
    assert en.MeshEnergy(mp).energy(xm) == pytest.approx(en.WarpEnergy(wp).energy(xw.reshape(-1)), rel=1e-12)


@pytest.mark.parametrize("mask_frac", [0.0, 0.3])
def test_warp_on_explicit_graph_equals_grid_warp(mask_frac):
    # The explicit-graph form of the warp (Fig. 18's comparison) has the grid
    # energy's residuals in another order: equal E, J^T F and J^T J.
    wp = tiny_warp(W=6, H=5, n_handles=4, seed=21, mask_frac=mask_frac, noise=0.4)
    if mask_frac:
        wp.handle_idx[0] = int(np.flatnonzero(wp.mask.reshape(-1))[0])   # a handle on a masked pixel is dropped
    gp = synth.warp_graph_from_grid(wp)
    eg, ew = en.make_energy(gp), en.WarpEnergy(wp)
    x = wp.x0.reshape(-1).astype(np.float64) + np.random.default_rng(2).uniform(-0.3, 0.3, wp.n_unknowns)
    assert eg.energy(x) == pytest.approx(ew.energy(x), rel=1e-13)
    Jg, Jw = eg.jacobian(x), ew.jacobian(x)
    np.testing.assert_allclose(Jg.T @ eg.residuals(x), Jw.T @ ew.residuals(x), rtol=0, atol=1e-11)
    np.testing.assert_allclose((Jg.T @ Jg).toarray(), (Jw.T @ Jw).toarray(), rtol=0, atol=1e-11)


def test_warp_graph_rigid_motion_has_zero_regularizer():
    # O = R(phi) U + t with theta = phi on every vertex: every edge residual vanishes
    rng = np.random.default_rng(4)
    V = 9
    U = rng.uniform(-3, 3, (2, V)).astype(np.float32)
    a = rng.integers(0, V, 30)
    b = (a + rng.integers(1, V, 30)) % V
    order = np.lexsort((b, a))
    phi, t = 0.7, np.array([[1.5], [-0.25]])
    O = en.rot2d(phi) @ U.astype(np.float64) + t
    gp = synth.WarpGraphProblem(V=V, urshape=U, v0=a[order].astype(np.int32), v1=b[order].astype(np.int32),
                                x0=np.zeros((3, V), np.float32), handle_idx=np.zeros(0, np.int32),
                                handle_target=np.zeros((0, 2), np.float32))
    x = np.concatenate([O - U, np.full((1, V), phi)]).reshape(-1)
    assert en.make_energy(gp).energy(x) == pytest.approx(0.0, abs=1e-20)


def test_volume_stencil_count_and_equals_mesh_on_the_voxel_graph():
    # Fig. 31: the 7-point stencil on a W x H x D array; as an explicit graph of
    # the same neighbour pairs it is the Fig. 25 energy (Rotate3D at the centre)
    W, H, D = 4, 3, 5
    vp = synth.volume_problem(W, H, D, 6, seed=2, x0_noise=0.3)
    ev = en.make_energy(vp)
    assert ev.a.size == 2 * ((W - 1) * H * D + W * (H - 1) * D + W * H * (D - 1))
    v0, v1 = synth.volume_edges(W, H, D)
    em = en.MeshEnergy(synth.MeshProblem(vp.V, vp.urshape, v0, v1, vp.x0, vp.handle_idx, vp.handle_target))
    x = vp.x0.reshape(-1).astype(np.float64) + np.random.default_rng(3).uniform(-0.2, 0.2, vp.n_unknowns)
    assert ev.energy(x) == pytest.approx(em.energy(x), rel=1e-13)
    Jv, Jm = ev.jacobian(x), em.jacobian(x)
    np.testing.assert_allclose(Jv.T @ ev.residuals(x), Jm.T @ em.residuals(x), rtol=0, atol=1e-11)
    np.testing.assert_allclose((Jv.T @ Jv).toarray(), (Jm.T @ Jm).toarray(), rtol=0, atol=1e-11)


def test_volume_rigid_motion_has_zero_regularizer():
    from scipy.spatial.transform import Rotation
    vp = synth.volume_problem(3, 4, 3, 1, seed=5)
    ang = np.array([0.3, -0.5, 0.9])
    R = Rotation.from_euler("xyz", ang).as_matrix()      # = Rz Ry Rx (extrinsic xyz)
    U = vp.urshape.astype(np.float64)
    O = R @ U + np.array([[1.0], [2.0], [-0.5]])
    x = np.concatenate([O - U, np.repeat(ang[:, None], vp.V, 1)]).reshape(-1)
    vp.handle_idx = np.zeros(0, np.int32)
    vp.handle_target = np.zeros((0, 3), np.float32)
    assert en.make_energy(vp).energy(x) == pytest.approx(0.0, abs=1e-18)


# --------------------------------------------------------------------------
# Jacobian: central finite differences; gradient = 2 J^T F
# --------------------------------------------------------------------------
# --------------------------------------------------------------------------
# embedded deformation (Fig. 28)
# --------------------------------------------------------------------------
def embedded_from(U, v0, v1, x, handle_idx=(), handle_target=None, w_rot=1.0):
    U = np.asarray(U, np.float32)
    hidx = np.asarray(handle_idx, np.int32)
    htgt = np.zeros((hidx.size, 3), np.float32) if handle_target is None else np.asarray(handle_target, np.float32)
    return synth.EmbeddedProblem(U.shape[1], U, np.asarray(v0, np.int32), np.asarray(v1, np.int32),
                                 np.asarray(x, np.float32), hidx, htgt, w_rot=w_rot)


def test_golden_embedded_2v():
    g = _golden("embedded_2v.json")
    prob = embedded_from(g["urshape"], g["v0"], g["v1"], g["x"])
    e = en.EmbeddedEnergy(prob)
    jtf, diag, E = so.jtf_diag(e, np.array(g["x"], np.float64).reshape(-1))
    assert E == pytest.approx(g["E"], abs=1e-12)
    np.testing.assert_allclose(jtf, np.array(g["jtf"]).reshape(-1), atol=1e-12)
    np.testing.assert_allclose(diag, np.array(g["diag"]).reshape(-1), atol=1e-12)


def test_embedded_rest_state_and_fit_closed_form():
    prob = synth.embedded_problem(1, seed=3)
    e = en.EmbeddedEnergy(prob)
    t = prob.handle_target.astype(np.float64)
    assert e.energy(prob.x0.reshape(-1)) == pytest.approx(prob.w_fit * float((t * t).sum()), rel=1e-13)
    prob.handle_target[:] = 0
    jtf, _, E = so.jtf_diag(en.EmbeddedEnergy(prob), prob.x0.reshape(-1))
    assert E == 0.0 and np.abs(jtf).max() == 0.0


def test_embedded_rigid_motion_is_free_and_scaling_closed_form():
    prob = synth.embedded_problem(2, seed=4, w_rot=2.5)
    prob.handle_idx = prob.handle_idx[:0]
    prob.handle_target = prob.handle_target[:0]
    e = en.EmbeddedEnergy(prob)
    U = prob.urshape.astype(np.float64)
    Q = Rotation.from_euler("zyx", [0.7, -0.4, 1.9]).as_matrix()
    O = Q @ U + np.array([[0.5], [1.0], [-2.0]])
    x = np.concatenate([(O - U).reshape(-1), np.repeat(Q.reshape(-1), prob.V)])
    assert e.energy(x) < 1e-20
    # R = s I, O = U: edge residuals (1 - s)(U_a - U_b), three constraints s^2 - 1 per vertex
    s_ = 1.3
    x2 = np.concatenate([np.zeros(3 * prob.V), np.repeat((s_ * np.eye(3)).reshape(-1), prob.V)])
    dU = U[:, prob.v0] - U[:, prob.v1]
    ref = prob.w_reg * (1 - s_) ** 2 * float((dU * dU).sum()) + prob.w_rot * prob.V * 3 * (s_ * s_ - 1) ** 2
    assert e.energy(x2) == pytest.approx(ref, rel=1e-12)


def test_embedded_constraints_act_on_columns():
    """The six constraints use the columns of R (Fig. 28 builds c0 from
    R(0), R(3), R(6)).  For R = [[1,1,1],[0,1,0],[0,0,1]] the column dots are
    (1, 1, 1) and the squared column norms (1, 2, 2): E = w_rot (3 + 0 + 1 + 1)
    = 5 w_rot (the rows would give 6 w_rot)."""
    R = np.array([[1.0, 1.0, 1.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    x = np.concatenate([np.zeros(3), R.reshape(-1)]).reshape(12, 1)
    prob = embedded_from(np.zeros((3, 1)), [], [], x, w_rot=0.7)
    assert en.EmbeddedEnergy(prob).energy(x.reshape(-1)) == pytest.approx(5 * 0.7, rel=1e-14)


def test_embedded_with_rotation_matrices_equals_arap_mesh():
    """With R_v the rotation Rz Ry Rx(A_v) the edge term is the ARAP mesh
    residual and the column constraints vanish: the two energies agree."""
    m = synth.mesh_problem(1, seed=9, handle_frac=0.2, x0_noise=0.4)
    ed = synth.embedded_problem(1, seed=9, handle_frac=0.2)
    x_mesh = m.x0.reshape(-1).astype(np.float64)
    A = m.x0[3:6].astype(np.float64)
    R, _ = en.euler_rotation(A.T)                            # (V, 3, 3)
    x_ed = np.concatenate([m.x0[0:3].astype(np.float64).reshape(-1),
                           np.transpose(R, (1, 2, 0)).reshape(-1)])
    Em = en.MeshEnergy(m).energy(x_mesh)
    Ee = en.EmbeddedEnergy(ed).energy(x_ed)
    assert Ee == pytest.approx(Em, rel=1e-12)


def random_warp_graph(seed=6):
    rng = np.random.default_rng(seed)
    V = 7
    a = rng.integers(0, V, 16)
    b = (a + rng.integers(1, V, 16)) % V
    order = np.lexsort((b, a))
    return synth.WarpGraphProblem(V=V, urshape=rng.uniform(-2, 2, (2, V)).astype(np.float32),
                                  v0=a[order].astype(np.int32), v1=b[order].astype(np.int32),
                                  x0=rng.uniform(-0.5, 0.5, (3, V)).astype(np.float32),
                                  handle_idx=np.array([1, 4], np.int32),
                                  handle_target=rng.uniform(-1, 1, (2, 2)).astype(np.float32))


@pytest.mark.parametrize("make", [
    lambda: (tiny_warp(), None),
    lambda: (tiny_warp(mask_frac=0.3, seed=9), None),
    lambda: (tiny_mesh(), None),
    lambda: (synth.poisson_problem(6, 5, seed=2), None),
    lambda: (random_warp_graph(), None),
    lambda: (synth.volume_problem(3, 2, 3, 2, seed=4, x0_noise=0.3), None),
    lambda: (synth.embedded_problem(0, seed=5, handle_frac=0.2, x0_noise=0.3), None),
])
def test_jacobian_matches_central_differences(make):
    prob, _ = make()
    e = en.make_energy(prob)
    rng = np.random.default_rng(1)
    x = prob.x0.reshape(-1).astype(np.float64) + rng.uniform(-0.2, 0.2, prob.n_unknowns)
    if prob.kind == "poisson":
        x = x.reshape(4, -1)
        x[:, prob.mask.reshape(-1) != 0] = prob.x0.reshape(4, -1)[:, prob.mask.reshape(-1) != 0]
        x = x.reshape(-1)
    J = e.jacobian(x).toarray()
    Jfd = fd_jacobian(e, x)
    if prob.kind == "poisson":       # fixed pixels are not unknowns: zero columns
        fixed = np.tile(prob.mask.reshape(-1) != 0, 4)
        Jfd[:, fixed] = 0.0
    scale = max(1.0, np.abs(J).max())
    assert np.abs(J - Jfd).max() <= 1e-7 * scale


def test_gradient_is_twice_jtf():
    prob = tiny_mesh(seed=12)
    e = en.MeshEnergy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    jtf, _, _ = so.jtf_diag(e, x)
    h = 1e-6
    g = np.array([(e.energy(x + h * np.eye(x.size)[i]) - e.energy(x - h * np.eye(x.size)[i])) / (2 * h)
                  for i in range(x.size)])
    np.testing.assert_allclose(g, 2 * jtf, atol=1e-6 * max(1.0, np.abs(g).max()))


# --------------------------------------------------------------------------
# J^T J: symmetry, PSD, closed-form stencils, null space, diagonals
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["warp", "mesh", "poisson", "embedded"])
def test_jtj_symmetric_psd_and_matrix_free_equals_dense(kind):
    prob = {"warp": lambda: tiny_warp(5, 4, 3, seed=21),
            "mesh": lambda: tiny_mesh(seed=22),
            "embedded": lambda: synth.embedded_problem(0, seed=24, handle_frac=0.2, x0_noise=0.3),
            "poisson": lambda: synth.poisson_problem(7, 6, seed=23)}[kind]()
    e = en.make_energy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    J = e.jacobian(x).toarray()
    A = J.T @ J
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() >= -1e-12 * np.abs(A).max()
    p = np.random.default_rng(0).standard_normal(x.size)
    np.testing.assert_allclose(so.apply_jtj(e, x, p), A @ p, rtol=1e-12, atol=1e-12)


def test_poisson_interior_stencil_closed_form():
    # interior free pixel with four free neighbours: q_i = 8 p_i - 2 sum p_nbr
    W, H = 9, 8
    mask = np.ones((H, W), np.uint8)
    mask[1:7, 1:8] = 0
    prob = synth.poisson_problem(W, H, seed=3, mask=mask)
    e = en.PoissonEnergy(prob)
    p = np.random.default_rng(2).standard_normal(4 * W * H)
    p.reshape(4, H, W)[:, mask != 0] = 0.0          # fixed pixels carry no unknown
    q = so.apply_jtj(e, prob.x0.reshape(-1), p).reshape(4, H, W)
    P = p.reshape(4, H, W)
    for y in range(2, 6):
        for x in range(2, 7):
            ref = 8 * P[:, y, x] - 2 * (P[:, y, x + 1] + P[:, y, x - 1] + P[:, y + 1, x] + P[:, y - 1, x])
            np.testing.assert_allclose(q[:, y, x], ref, atol=1e-12)


def test_warp_translation_null_space_and_diag_closed_form():
    W, H = 6, 5
    prob = synth.warp_problem(W, H, 0, seed=31, x0_noise=0.5)
    prob.w_reg = 1.7
    e = en.WarpEnergy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    p = np.concatenate([np.full(W * H, 0.3), np.full(W * H, -1.2), np.zeros(W * H)])
    assert np.abs(so.apply_jtj(e, x, p)).max() < 1e-12
    # diag: O rows = w_reg * 2 * #valid neighbours (+ w_fit at handles);
    # theta rows = w_reg * sum_d |R'(theta) v|^2 = w_reg * sum_d |v|^2 = w_reg * #valid
    prob2 = synth.warp_problem(W, H, 4, seed=32, x0_noise=0.5)
    prob2.w_reg = 1.7
    _, diag, _ = so.jtf_diag(en.WarpEnergy(prob2), prob2.x0.reshape(-1))
    nb = np.zeros((H, W))
    nb[:, :-1] += 1
    nb[:, 1:] += 1
    nb[:-1, :] += 1
    nb[1:, :] += 1
    hfit = np.zeros(W * H)
    hfit[prob2.handle_idx] = prob2.w_fit
    np.testing.assert_allclose(diag[:W * H], 1.7 * 2 * nb.reshape(-1) + hfit, rtol=1e-13)
    np.testing.assert_allclose(diag[W * H:2 * W * H], 1.7 * 2 * nb.reshape(-1) + hfit, rtol=1e-13)
    np.testing.assert_allclose(diag[2 * W * H:], 1.7 * nb.reshape(-1), rtol=1e-12)


# --------------------------------------------------------------------------
# PCG: exact in n steps, recurrence residual, monotone quadratic model
# --------------------------------------------------------------------------
def test_pcg_matches_dense_solve_and_is_monotone():
    prob = tiny_warp(3, 3, 3, seed=41, noise=0.4)
    e = en.WarpEnergy(prob)
    x = prob.x0.reshape(-1).astype(np.float64)
    J = e.jacobian(x).toarray()
    A = J.T @ J
    assert np.linalg.eigvalsh(A).min() > 0                       # SPD with handles
    b = -(J.T @ e.residuals(x))
    Minv = so.jacobi_minv(np.diag(A).copy())
    n = A.shape[0]
    d, n_done, r = so.jacobi_pcg(lambda p: A @ p, b, Minv, n)
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(d - ref) <= 1e-9 * np.linalg.norm(ref)
    # quadratic model m(d) = 1/2 d^T A d - b^T d decreases every iteration;
    # the recurrence residual equals b - A d
    prev = 0.0
    for k in range(1, 12):
        dk, _, rk = so.jacobi_pcg(lambda p: A @ p, b, Minv, k)
        m = 0.5 * dk @ A @ dk - b @ dk
        assert m <= prev + 1e-12 * abs(prev)
        prev = m
        np.testing.assert_allclose(rk, b - A @ dk, atol=1e-9 * np.linalg.norm(b))


def test_pcg_stops_on_zero_rhs():
    d, n_done, _ = so.jacobi_pcg(lambda p: 2 * p, np.zeros(5), np.ones(5), 10)
    assert n_done == 0 and not d.any()


# --------------------------------------------------------------------------
# GN: exact for linear problems (Sec. 8.1); LM: monotone, limits
# --------------------------------------------------------------------------
def test_gn_poisson_one_step_reaches_least_squares_optimum():
    prob = synth.poisson_problem(8, 7, seed=51)
    e = en.PoissonEnergy(prob)
    x0 = prob.x0.reshape(-1).astype(np.float64)
    free = np.tile(prob.mask.reshape(-1) == 0, 4)
    n = int(free.sum())
    res = so.gauss_newton(e, x0, outer=2, inner=n + 5)
    J = e.jacobian().toarray()[:, free]
    dref = np.linalg.lstsq(J, -e.residuals(x0), rcond=None)[0]
    xref = x0.copy()
    xref[free] += dref
    np.testing.assert_allclose(res.x, xref, atol=1e-9)
    jtf, _, _ = so.jtf_diag(e, res.x)
    assert np.abs(jtf).max() < 1e-9
    assert res.E_history[1] == pytest.approx(res.E_history[2], rel=1e-10, abs=1e-14)


def test_gn_nonlinear_step_is_dense_normal_equation_solve():
    prob = tiny_warp(4, 4, 3, seed=52, noise=0.3)
    e = en.WarpEnergy(prob)
    x0 = prob.x0.reshape(-1).astype(np.float64)
    res = so.gauss_newton(e, x0, outer=1, inner=e.N + 10)
    J = e.jacobian(x0).toarray()
    d = np.linalg.solve(J.T @ J, -J.T @ e.residuals(x0))
    np.testing.assert_allclose(res.x, x0 + d, atol=1e-8)


def test_lm_energy_monotone_over_accepted_steps():
    prob = synth.mesh_problem(2, seed=61, handle_frac=0.1)
    e = en.MeshEnergy(prob)
    res = so.levenberg_marquardt(e, prob.x0.reshape(-1), outer=8, inner=20)
    E = res.E_history
    for k, acc in enumerate(res.accepted):
        if acc:
            assert E[k + 1] <= E[k] * (1 + 1e-12)
        else:
            assert E[k + 1] == E[k]
    assert E[-1] < E[0]


def test_lm_small_lambda_is_gn_and_large_lambda_is_scaled_gradient():
    prob = tiny_warp(4, 3, 3, seed=62, noise=0.2)
    e = en.WarpEnergy(prob)
    x0 = prob.x0.reshape(-1).astype(np.float64)
    n = e.N + 10
    gn = so.gauss_newton(e, x0, outer=1, inner=n)
    lm = so.levenberg_marquardt(e, x0, outer=1, inner=n,
                                prm=so.LMParams(lambda0=1e-14, lambda_min=1e-20))
    if lm.accepted[0]:
        np.testing.assert_allclose(lm.x, gn.x, atol=1e-7)
    # large damping: (J^T J + lam Dc) d = b  ->  d ~ b / (lam Dc)
    J = e.jacobian(x0)
    F = e.residuals(x0)
    b = -(J.T @ F)
    diag = np.asarray(J.multiply(J).sum(0)).ravel()
    Dc = np.clip(diag, 1e-6, 1e32)
    lam = 1e8
    d, _, _ = so.jacobi_pcg(lambda p: J.T @ (J @ p) + lam * Dc * p, b,
                            so.jacobi_minv(diag + lam * Dc), 50)
    np.testing.assert_allclose(d, b / (lam * Dc), rtol=1e-6, atol=1e-14)


def test_lm_linear_problem_gain_ratio_is_one():
    # For a linear problem the linear model is exact, so the gain ratio is 1
    # and Nielsen's update divides lambda by max(3, 1/(1 - (2*1-1)^3)) = 3.
    prob = synth.poisson_problem(8, 7, seed=71)
    e = en.PoissonEnergy(prob)
    n = int((prob.mask == 0).sum()) * 4 + 5
    res = so.levenberg_marquardt(e, prob.x0.reshape(-1), outer=3, inner=n,
                                 prm=so.LMParams(lambda0=0.5))
    assert res.accepted[:2] == [True, True]
    assert res.lambdas[1] == pytest.approx(0.5 / 3, rel=1e-12)
    assert res.lambdas[2] == pytest.approx(0.5 / 9, rel=1e-12)


def test_lm_rejections_double_nu():
    # eta above any attainable gain ratio rejects every step: lambda grows by
    # nu = 2, 4, 8 (cumulative factors 2, 8, 64) and x never moves.
    prob = synth.poisson_problem(8, 7, seed=72)
    e = en.PoissonEnergy(prob)
    res = so.levenberg_marquardt(e, prob.x0.reshape(-1), outer=4, inner=10,
                                 prm=so.LMParams(lambda0=1e-3, eta=2.0))
    assert res.accepted == [False] * 4
    np.testing.assert_allclose(res.lambdas, [1e-3, 2e-3, 8e-3, 64e-3], rtol=1e-12)
    np.testing.assert_array_equal(res.x, prob.x0.reshape(-1).astype(np.float64))


def test_lm_large_damping_step_is_scaled_gradient_through_solver():
    # (J^T J + lam Dc) d = b with lam -> inf gives d -> b / (lam Dc); for the
    # warp the diagonal has the closed form pinned above.
    W, H = 6, 5
    prob = synth.warp_problem(W, H, 3, seed=73, x0_noise=0.05)
    e = en.WarpEnergy(prob)
    x0 = prob.x0.reshape(-1).astype(np.float64)
    jtf, diag, _ = so.jtf_diag(e, x0)
    lam = 1e7
    res = so.levenberg_marquardt(e, x0, outer=1, inner=30, prm=so.LMParams(lambda0=lam))
    assert res.accepted == [True]
    ref = -jtf / (lam * np.clip(diag, 1e-6, 1e32))
    assert np.linalg.norm(res.x - x0 - ref) <= 1e-5 * np.linalg.norm(ref)


def test_damped_apply_matches_exact_lm_step():
    # An exact LM step d solves (J^T J + lam Dc) d = -J^T F, which ties the
    # damped matrix-free product to the (pinned) LM routine.
    prob = synth.poisson_problem(7, 6, seed=74)
    e = en.PoissonEnergy(prob)
    x0 = prob.x0.reshape(-1).astype(np.float64)
    n = int((prob.mask == 0).sum()) * 4 + 5
    lam = 0.5
    res = so.levenberg_marquardt(e, x0, outer=1, inner=n, prm=so.LMParams(lambda0=lam))
    assert res.accepted == [True]
    jtf, diag, _ = so.jtf_diag(e, x0)
    q = so.apply_jtj(e, x0, res.x - x0, lam, np.clip(diag, 1e-6, 1e32))
    np.testing.assert_allclose(q, -jtf, atol=1e-9 * np.abs(jtf).max())


# -- reduced-precision storage emulation (round_to) -------------------------------

def test_round_to_none_is_the_plain_run():
    prob = synth.mesh_problem(1, seed=21, handle_frac=0.2)
    e = en.make_energy(prob)
    x0 = prob.x0.reshape(-1)
    a = so.levenberg_marquardt(e, x0, 4, 8)
    b = so.levenberg_marquardt(e, x0, 4, 8, round_to=None)
    assert a.E_history == b.E_history and np.array_equal(a.x, b.x)
    g = so.gauss_newton(e, x0, 3, 6)
    h = so.gauss_newton(e, x0, 3, 6, round_to=None)
    assert g.E_history == h.E_history


def test_round_to_float32_stores_float32_values_and_stays_close_when_well_conditioned():
    """The emulated run keeps the state representable in float32; on a linear,
    well-conditioned problem (Poisson) its energies stay within float32
    rounding of the plain run, and LM stays monotone over accepted steps."""
    prob = synth.poisson_problem(24, 20, seed=23)
    e = en.make_energy(prob)
    x0 = prob.x0.reshape(-1)
    plain = so.gauss_newton(e, x0, 3, 15)
    f32 = so.gauss_newton(e, x0, 3, 15, round_to=np.float32)
    assert np.array_equal(f32.x, f32.x.astype(np.float32).astype(np.float64))
    for a, b in zip(f32.E_history, plain.E_history):
        assert abs(a - b) <= 1e-5 * b
    m = synth.mesh_problem(1, seed=24, handle_frac=0.2)
    em = en.make_energy(m)
    lm = so.levenberg_marquardt(em, m.x0.reshape(-1), 6, 10, round_to=np.float32)
    acc_E = [lm.E_history[0]] + [lm.E_history[k + 1] for k, a in enumerate(lm.accepted) if a]
    assert all(b <= a for a, b in zip(acc_E, acc_E[1:]))
    assert np.array_equal(lm.x, lm.x.astype(np.float32).astype(np.float64))
