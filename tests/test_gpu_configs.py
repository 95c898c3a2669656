"""Parity at each workload's stated size, through the C ABI, against the FP64 oracle.

- C1: 160x120, ~20k triangles, sigma 1 cm, 5% dropout: one cost evaluation, then LM from
  5 cm / 2 deg to the oracle's pose within 1 mm / 0.01 deg.
- C2: 640x480 Kinect camera, ~500k triangles (20% FU interfaces), noise 0.5% of depth:
  cost and adjoint gradient against the oracle's FP64 values, against central finite
  differences at h = 1e-4 of the oracle's frozen-visibility cost, and through the
  torch.autograd.Function (RenderMapCost) backward.
- C3: 256 candidate poses (10 cm / 5 deg) at 320x240 on the 1M-triangle room, all in one
  persistent launch (and in waves): every pose against the oracle.
- C4: 1024x64 panoramic Lidar on the 2M-triangle terrain: LM from 30 cm / 3 deg lands within
  1 mm / 0.01 deg of the oracle's LM.
- C5: the 64-agent mixed-sensor tracking batch on the 2M-triangle terrain, 5 LM iterations
  per agent in one persistent launch: on two sampled frames, every agent's iterations equal
  the single-problem LM's bit for bit, and each one lands where one oracle LM iteration from
  the same iterate and damping lands.

Tolerances: Table I counts bit for bit, E_ls 1e-5 relative, gradients and J^T J 1e-3
element by element (tests/checks.py), poses 1 mm / 0.01 deg.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import cases
import checks
import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker is deselected on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1702_06813_gb300 as rm  # noqa: E402
from paper_1702_06813_gb300 import build as rmbuild  # noqa: E402

rmbuild.build()

EPS_REL_COST = 1e-5
EPS_REL_GRAD = 1e-3
POOL = ThreadPoolExecutor(max_workers=os.cpu_count() or 4)  # the oracle's C calls drop the GIL


def _np(t):
    return t.detach().cpu().numpy() if torch.is_tensor(t) else np.asarray(t)


def _pose_gap(a, b):
    dt = float(np.linalg.norm(a[:3, 3] - b[:3, 3]))
    da = math.degrees(Rotation.from_matrix(a[:3, :3].T @ b[:3, :3]).magnitude())
    return dt, da


def _check_cost(g, k, o, grad=True, what=""):
    assert np.array_equal(_np(g["counts"])[k], o["counts"]), (what, k)
    assert int(_np(g["e_table"])[k]) == int(o["counts"][1] + o["counts"][3] + o["counts"][5]
                                            - o["counts"][0] - o["counts"][2] - o["counts"][4])
    e = float(_np(g["e_ls"])[k])
    assert abs(e - o["e_ls"]) <= EPS_REL_COST * abs(o["e_ls"]) + 1e-12, (what, k, e, o["e_ls"])
    if grad:
        checks.close_elementwise(_np(g["grad"])[k], o["grad"], EPS_REL_GRAD, f"{what}_grad[{k}]", floor=1e-9)
        checks.close_elementwise(_np(g["jtj"])[k], o["jtj"], EPS_REL_GRAD, f"{what}_jtj[{k}]", floor=1e-9)


def _batch_rows(b, k):
    return {"counts": b["counts"][k], "e_ls": b["e_ls"][k], "grad": b["grad"][k], "jtj": b["jtj"][k]}


# ---------------------------------------------------------------------------------------
# C1
# ---------------------------------------------------------------------------------------

def test_c1_cost_then_lm():
    c = cases.config1(seed=1000)
    mesh, cam = c["mesh"], c["cam"]
    assert 19_000 <= mesh.n_tris <= 21_000
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(cam), *c["scan"])
    g = rm.cost_grad(gm, scan, c["start"][None])
    _check_cost(g, 0, om.cost(c["start"], cam, *c["scan"]), what="c1")
    pg, rep = rm.align(gm, scan, c["start"], max_iters=50, step_tol=1e-7)
    po, orep = om.align(c["start"], cam, *c["scan"], max_iters=50, step_tol=1e-7)
    dt, da = _pose_gap(pg, po)
    assert dt < 1e-3 and da < 1e-2, (dt, da, rep, orep)
    gm.close()


# ---------------------------------------------------------------------------------------
# C2
# ---------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def c2():
    c = cases.config2()  # 400k FO + 100k FU triangles, 640x480, noise 0.5% of depth
    mesh, cam = c["mesh"], c["cam"]
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(cam), *c["scan"])
    yield dict(c, om=om, gm=gm, gscan=scan)
    gm.close()


def test_c2_size(c2):
    mesh = c2["mesh"]
    assert 475_000 <= mesh.n_tris <= 525_000
    fu = float(np.mean(mesh.labels == 1))
    assert 0.18 <= fu <= 0.22, fu
    assert (c2["cam"].width, c2["cam"].height, c2["cam"].fx) == (640, 480, 525.0)


def test_c2_cost_and_gradient_against_oracle(c2):
    r = cases.rng(2101)
    poses = [c2["gt"], c2["start"]] + [synth.perturb_fixed(c2["gt"], r, 0.1, 3.0) for _ in range(2)]
    g = rm.cost_grad(c2["gm"], c2["gscan"], np.stack(poses))
    outs = list(POOL.map(lambda P: c2["om"].cost(P, c2["cam"], *c2["scan"]), poses))
    for k, o in enumerate(outs):
        _check_cost(g, k, o, what="c2")
    # every Table I outcome of the FU interfaces shows up
    assert np.all(_np(g["counts"]).sum(0)[[0, 1, 4, 5]] > 0)


def test_c2_gradient_against_central_fd_h1e4(c2):
    """Central differences (h = 1e-4) of the oracle's FP64 frozen-visibility cost, the
    quantity the adjoint differentiates."""
    P = c2["start"]
    g = _np(rm.cost_grad(c2["gm"], c2["gscan"], P[None])["grad"])[0]
    h = 1e-4

    def fd(a):
        xi = np.zeros(6)
        xi[a] = h
        return (c2["om"].cost_frozen(P, c2["cam"], *c2["scan"], xi)
                - c2["om"].cost_frozen(P, c2["cam"], *c2["scan"], -xi)) / (2 * h)

    d = np.array(list(POOL.map(fd, range(6))))
    checks.close_elementwise(g, d, EPS_REL_GRAD, "c2_grad_vs_fd_h1e-4")


def test_c2_autograd_backward(c2):
    """RenderMapCost (torch.autograd.Function): forward equals the oracle's E_ls at the
    retracted pose; backward equals the chain rule J_r(xi)^T grad of the oracle, and central
    differences (h = 1e-4) of the oracle's frozen cost in xi."""
    P = c2["start"]
    xi0 = np.array([0.004, -0.006, 0.003, 0.002, -0.001, 0.003])
    xi = torch.tensor(xi0, dtype=torch.float64, requires_grad=True)
    e = rm.RenderMapCost.apply(xi, P, c2["gm"], c2["gscan"], None)
    e.backward()
    Pr = oracle.se3_right(P, xi0)
    o = c2["om"].cost(Pr, c2["cam"], *c2["scan"])
    assert abs(e.item() - o["e_ls"]) <= EPS_REL_COST * o["e_ls"]
    _, jr = rm.pose_retract(P[None], xi0[None], with_jacobian=True)
    checks.close_elementwise(_np(xi.grad), _np(jr[0]).T @ o["grad"], EPS_REL_GRAD, "c2_autograd")
    # the same derivative by differences in xi, through the frozen cost at P exp(xi +- h e_a)
    h = 1e-4

    def fd(a):
        d = np.zeros(6)
        d[a] = h
        # frozen cells of the retracted pose; the perturbation is applied on the right of it
        Jp = oracle.se3_right(np.eye(4), xi0 + d)
        Jm = oracle.se3_right(np.eye(4), xi0 - d)
        E0 = oracle.se3_right(np.eye(4), xi0)
        xp = _log_se3(np.linalg.inv(E0) @ Jp)
        xm = _log_se3(np.linalg.inv(E0) @ Jm)
        return (c2["om"].cost_frozen(Pr, c2["cam"], *c2["scan"], xp)
                - c2["om"].cost_frozen(Pr, c2["cam"], *c2["scan"], xm)) / (2 * h)

    d = np.array(list(POOL.map(fd, range(6))))
    checks.close_elementwise(_np(xi.grad), d, EPS_REL_GRAD, "c2_autograd_vs_fd")


def _log_se3(T):
    """Twist (rho, phi) with se3_right(I, xi) == T (small rotations; inverse of the SE(3)
    exponential by the left Jacobian's inverse)."""
    R = T[:3, :3]
    phi = Rotation.from_matrix(R).as_rotvec()
    th = np.linalg.norm(phi)
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    if th < 1e-12:
        Jinv = np.eye(3) - 0.5 * K
    else:
        a = (1 - th * math.sin(th) / (2 * (1 - math.cos(th)))) / th ** 2
        Jinv = np.eye(3) - 0.5 * K + a * K @ K
    return np.concatenate([Jinv @ T[:3, 3], phi])


# ---------------------------------------------------------------------------------------
# C3
# ---------------------------------------------------------------------------------------

def test_c3_256_poses_320x240_persistent_and_waves():
    w = synth.workload_headline(3000, 256)  # 800k FO + 200k FU; poses 10 cm / 5 deg around GT
    mesh = w["mesh"]
    assert 990_000 <= mesh.n_tris <= 1_010_000
    cam = synth.cam_320x240()
    scan_np = synth.synth_scan(mesh, cam, w["gt"], cases.rng(3301), sigma_rel=0.005)
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(cam), *scan_np)
    poses = torch.as_tensor(w["poses"].reshape(-1, 16), dtype=torch.float64, device="cuda")
    b = rm.cost_grad_batch(gm, scans=scan, poses=poses)   # one persistent launch (CUDA graph)
    waves = rm.cost_grad(gm, scan, poses)
    o = om.cost_batch(w["poses"], cam, *scan_np)
    for k in range(256):
        ok = {"counts": o["counts"][k], "e_ls": o["e_ls"][k], "grad": o["grad"][k], "jtj": o["jtj"][k]}
        _check_cost(b, k, ok, what="c3")
    for key in ("counts", "e_table", "e_ls", "grad", "jtj"):
        assert torch.equal(b[key], waves[key]), key
    gm.close()


# ---------------------------------------------------------------------------------------
# C4, C5: the 2M-triangle terrain
# ---------------------------------------------------------------------------------------

def test_c4_lidar_lm_full_size():
    w = synth.workload_lidar()  # 1.4M FO + 0.6M FU, 1024x64, sigma 2 cm, start 30 cm / 3 deg
    mesh, cam = w["mesh"], w["cam"]
    assert 1_900_000 <= mesh.n_tris <= 2_100_000
    fu = float(np.mean(mesh.labels == 1))
    assert 0.27 <= fu <= 0.33, fu
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(cam), *w["scan"])
    pg, rep = rm.align(gm, scan, w["start"], max_iters=200, step_tol=1e-7)
    po, orep = om.align(w["start"], cam, *w["scan"], max_iters=200, step_tol=1e-7)
    dt, da = _pose_gap(pg, po)
    assert dt < 1e-3 and da < 1e-2, (dt, da, rep, orep)
    assert rep["e_ls_final"] < rep["e_ls_initial"]
    gm.close()


def _lm_step(P, g, H21, lam):
    """One LM proposal in FP64: (H + lam diag H) dx = -g, P exp(dx^) (the step both sides take)."""
    H = np.zeros((6, 6))
    k = 0
    for u in range(6):
        for v in range(u, 6):
            H[u, v] = H[v, u] = H21[k]
            k += 1
    A = H + lam * np.diag(np.diag(H))
    try:
        L = np.linalg.cholesky(A)  # the device solves by Cholesky: not positive definite = no step
    except np.linalg.LinAlgError:
        return None
    return oracle.se3_right(P, -np.linalg.solve(L.T, np.linalg.solve(L, g)))


def test_c5_tracking_batch_sampled_frames():
    """Two sampled frames of the tracking batch (64 agents, mixed sensors, 2M triangles). The
    batch's 5 LM iterations per agent equal the single-problem entry point's bit for bit, and
    every iteration is checked against the oracle from the GPU's own iterate k-1 and damping
    (lambda0 = 1e-3, divided by 10 on an accepted step, multiplied by 10 otherwise):
    - the cost, gradient and Gauss-Newton matrix at the iterate match the oracle's (counts
      exact, E_ls 1e-5, gradient and J^T J 1e-3 element by element; an element that misses
      that must lie within it plus the a-priori FP32 error bound of its sum, tests/checks.py
      fp32_bound: terrain seen from 1.5 m has grazing pixels whose n . r cancels);
    - the device's proposal is the FP64 LM step of those sums (within 1e-9 m / 1e-7 rad);
    - the accept decision equals the oracle's decision for the same proposal, unless the
      oracle's costs at the iterate and the proposal tie within the cost tolerance;
    - one oracle LM iteration from the same iterate and damping lands within 1 mm / 0.01 deg
      of the GPU's next iterate, or the two proposals differ only as the sums' tolerance
      allows: the LM solve amplifies the sums' differences by the damped system's condition
      number, which a single unconverged step from a poor start makes large.
    (Comparing only the fifth iterates would not be a parity test: from a poor start most pixels
    sit at the surrogate's truncation, and micrometres in one iterate change which pixels are
    inliers at the next, so two correct implementations part ways.)"""
    w = synth.workload_tracking(5000, n_agents=64, n_frames=200)
    mesh, cams, kinds, truth = w["mesh"], w["cams"], w["kinds"], w["poses"]
    assert 1_900_000 <= mesh.n_tris <= 2_100_000
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    fo = mesh.labels == 0
    om_fo = oracle.OracleMap(mesh.vertices, mesh.faces[fo], mesh.labels[fo])
    intr = [rm.Intrinsics.from_camera(c) for c in cams]
    n = truth.shape[1]
    K = 5
    far_steps = 0
    for f in (0, 120):
        r = cases.rng(5100 + f)
        starts = np.stack([synth.perturb_fixed(truth[f, a], r, 0.10, 1.0) for a in range(n)])
        noise = [r.normal(size=(cams[kinds[a]].height, cams[kinds[a]].width)) for a in range(n)]

        def scan_of(a):
            cam = cams[kinds[a]]
            d = om_fo.render(truth[f, a], cam)["depth"].astype(np.float64)
            sig = 0.02 if cam.model != "pinhole" else 0.005 * np.nan_to_num(d, nan=0.0)
            d = d + sig * noise[a]
            far = ~(d <= cam.range_max)
            d[far] = cam.range_max
            return d.astype(np.float32), far.astype(np.uint8)

        scans = list(POOL.map(scan_of, range(n)))
        gscans = [rm.Scan.make(intr[kinds[a]], *scans[a]) for a in range(n)]
        pb, reps, status = rm.align_batch(gm, [(gscans[a], starts[a]) for a in range(n)], max_iters=K)
        # the GPU's iterates 1..K of every agent (single-problem calls), dampings and sums
        iters = []
        for a in range(n):
            P, lam, acc, seq = starts[a], 1e-3, 0, []
            for k in range(1, K + 1):
                Pk, rk = rm.align(gm, gscans[a], starts[a], max_iters=k)
                if rk["converged"]:
                    break
                took = rk["accepted"] - acc
                g = rm.cost_grad(gm, gscans[a], P[None])
                seq.append((P, lam, Pk, took, {key: _np(v)[0] for key, v in g.items()}))
                lam = lam / 10.0 if took else lam * 10.0
                P, acc = Pk, rk["accepted"]
            assert np.array_equal(pb[a], P), a  # batch = single calls, bit for bit
            iters.append(seq)

        def oracle_steps(a):
            cam = cams[kinds[a]]
            out = []
            for (P, lam, Pk, took, gs) in iters[a]:
                o = om.cost(P, cam, *scans[a])
                prop = _lm_step(P, gs["grad"], gs["jtj"], lam)  # the GPU's proposal, recomputed
                e_prop = om.cost(prop, cam, *scans[a])["e_ls"] if prop is not None else None
                po, orep = om.align(P, cam, *scans[a], max_iters=1, lambda0=lam)
                out.append((o, gs, prop, e_prop, po, orep["accepted"], Pk, took))
            return out

        for a, steps in enumerate(POOL.map(oracle_steps, range(n))):
            cam = cams[kinds[a]]
            for k, (o, gs, prop, e_prop, po, oacc, Pk, took) in enumerate(steps):
                what = f"c5_f{f}_a{a}_k{k}"
                _check_cost({key: v[None] for key, v in gs.items()}, 0, o, grad=False, what="c5")
                P = iters[a][k][0]
                bound = {}

                def fp32(i, P=P, cam=cam, sc=scans[a]):
                    if not bound:
                        bound["b"] = checks.fp32_bound(om, P, cam, *sc)
                    return bound["b"][i]

                checks.close_elementwise_or_bounded(gs["grad"], o["grad"], EPS_REL_GRAD, f"c5_grad[{what}]",
                                                    lambda: fp32(0), floor=1e-9)
                checks.close_elementwise_or_bounded(gs["jtj"], o["jtj"], EPS_REL_GRAD, f"c5_jtj[{what}]",
                                                    lambda: fp32(1), floor=1e-9)
                if prop is None:  # no positive definite system: no step on either side
                    assert not took and oacc == 0, what
                    continue
                if took:  # the device's accepted pose is its proposal
                    dt, da = _pose_gap(Pk, prop)
                    assert dt < 1e-9 and da < 1e-7 * 180 / math.pi, (what, dt, da)
                else:
                    assert np.array_equal(Pk, iters[a][k][0]), what
                decided = e_prop < o["e_ls"]
                if decided != bool(took):
                    assert abs(e_prop - o["e_ls"]) <= 2 * EPS_REL_COST * o["e_ls"], (what, e_prop, o["e_ls"])
                    break  # a tie: the paths part here
                dt, da = _pose_gap(Pk, po)
                if not (dt < 1e-3 and da < 1e-2):
                    far_steps += 1
    # steps whose one-iteration poses differ beyond 1 mm / 0.01 deg (every one of them passed
    # the sums, solve and decision checks above)
    assert far_steps <= 0.05 * 2 * n * K, far_steps
    gm.close()
