"""The persistent batched form against the per-problem calls and the oracle.

A batch mixes camera models and sizes over one map. Each problem's result must equal what
rm_cost_grad / rm_align give for it alone, bit for bit (same kernels and reduction order), and
match the oracle within the parity tolerances.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import pytest

import cases
import checks
import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1702_06813_gb300 as rm  # noqa: E402
from paper_1702_06813_gb300 import build as rmbuild  # noqa: E402

rmbuild.build()


def _np(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def mixed():
    """Small terrain map seen by three sensor types (160x120 and 320x240 pinhole at 1.5 m,
    1024x64 Lidar at 1.8 m), noisy scans of the world, poses off the true ones."""
    mesh = synth.terrain_mesh(4200, target_fo=140_000, target_fu=60_000, n_panels=120)
    r = cases.rng(4201)
    cams = [dataclasses.replace(synth.cam_160x120(), range_max=40.0, near=0.3),
            dataclasses.replace(synth.cam_320x240(), range_max=40.0, near=0.3),
            synth.cam_lidar_1024x64()]
    probs = []
    for k in range(6):
        cam = cams[k % 3]
        gt = synth.terrain_pose(r, mesh, height=1.8 if cam.model == "spherical" else 1.5)
        if cam.model == "pinhole":  # look slightly down at the terrain
            gt = gt @ np.block([[synth.perturb(np.eye(4), np.zeros(3), np.array([-0.25, 0, 0]))[:3, :3],
                                 np.zeros((3, 1))], [np.zeros((1, 3)), np.ones((1, 1))]])
        sd, sc = synth.synth_scan(mesh, cam, gt, r, sigma_abs=0.02)
        start = synth.perturb_fixed(gt, r, 0.05 * (1 + k % 2), 1.0)
        probs.append(dict(cam=cam, gt=gt, scan=(sd, sc), start=start))
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    for pr in probs:
        pr["intr"] = rm.Intrinsics.from_camera(pr["cam"])
        pr["gscan"] = rm.Scan.make(pr["intr"], *pr["scan"])
    return dict(mesh=mesh, probs=probs, gm=gm, om=om)


def test_batch_cost_grad_equals_single_calls(mixed):
    gm = mixed["gm"]
    gm.set_tuning()  # default tiles: the batched kernel's per camera model
    b = rm.cost_grad_batch(gm, [(pr["gscan"], pr["start"]) for pr in mixed["probs"]])
    for k, pr in enumerate(mixed["probs"]):
        s = rm.cost_grad(gm, pr["gscan"], pr["start"][None])
        for key in ("counts", "e_table", "e_ls", "grad", "jtj"):
            assert torch.equal(b[key][k], s[key][0]), (k, key)
    # and one problem of each camera type against the oracle
    for k in range(3):
        pr = mixed["probs"][k]
        o = mixed["om"].cost(pr["start"], pr["cam"], *pr["scan"])
        assert np.array_equal(_np(b["counts"][k]), o["counts"])
        assert abs(float(b["e_ls"][k]) - o["e_ls"]) <= 1e-5 * abs(o["e_ls"])
        checks.close_elementwise(_np(b["grad"][k]), o["grad"], 1e-3, f"batch_grad[{k}]")
        checks.close_elementwise(_np(b["jtj"][k]), o["jtj"], 1e-3, f"batch_jtj[{k}]")


def test_batch_align_equals_single_calls(mixed):
    gm = mixed["gm"]
    gm.set_tuning()
    probs = mixed["probs"]
    poses, reps, status = rm.align_batch(gm, [(pr["gscan"], pr["start"]) for pr in probs], max_iters=5)
    for k, pr in enumerate(probs):
        ps, rs = rm.align(gm, pr["gscan"], pr["start"], max_iters=5)
        assert np.array_equal(poses[k], ps), k
        for f in ("iters", "accepted", "converged", "e_ls_final", "e_table_final"):
            assert reps[k][f] == rs[f], (k, f)
        assert reps[k]["e_ls_final"] <= reps[k]["e_ls_initial"]


def test_batch_many_problems_room():
    """40 candidate poses of the 160x120 room as a batch of independent problems."""
    c = cases.config1(seed=1000)
    gm = rm.Map(c["mesh"].vertices, c["mesh"].faces, c["mesh"].labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(c["cam"]), *c["scan"])
    r = cases.rng(44)
    poses = [synth.perturb_fixed(c["gt"], r, 0.1, 3.0) for _ in range(40)]
    b = rm.cost_grad_batch(gm, [(scan, P) for P in poses])
    s = rm.cost_grad(gm, scan, np.stack(poses))  # default tiles, as the batch
    for key in ("counts", "e_table", "e_ls", "grad", "jtj"):
        assert torch.equal(b[key], s[key]), key


def test_batch_repeated_calls_and_bin_growth():
    """Calls of one batch shape reuse the device queue: back-to-back calls with new poses, a
    per-pose call in between (which reuses the arena), and a call whose bins overflow and
    grow (which reallocates it) must all still equal the per-pose results."""
    c = cases.config1(seed=1000)
    gm = rm.Map(c["mesh"].vertices, c["mesh"].faces, c["mesh"].labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(c["cam"]), *c["scan"])
    r = cases.rng(45)
    A = np.stack([synth.perturb_fixed(c["gt"], r, 0.1, 3.0) for _ in range(24)])
    B = np.stack([synth.perturb_fixed(c["gt"], r, 0.1, 3.0) for _ in range(24)])
    keys = ("counts", "e_table", "e_ls", "grad", "jtj")
    bA = rm.cost_grad_batch(gm, scans=scan, poses=torch.as_tensor(A))
    bB = rm.cost_grad_batch(gm, scans=scan, poses=torch.as_tensor(B))  # same shape, new poses
    bB2 = rm.cost_grad_batch(gm, [(scan, P) for P in B])               # list form, same shape
    sA = rm.cost_grad(gm, scan, A)
    sB = rm.cost_grad(gm, scan, B)
    bA2 = rm.cost_grad_batch(gm, scans=scan, poses=torch.as_tensor(A))  # after a per-pose call
    for key in keys:
        assert torch.equal(bA[key], sA[key]), key
        assert torch.equal(bB[key], sB[key]), key
        assert torch.equal(bB2[key], sB[key]), key
        assert torch.equal(bA2[key], sA[key]), key
    gm.set_tuning(bin_capacity=4)  # every bin overflows: grown over several attempts
    bA3 = rm.cost_grad_batch(gm, scans=scan, poses=torch.as_tensor(A))
    assert gm.get_tuning()["bin_capacity"] > 4
    for key in keys:
        assert torch.equal(bA3[key], sA[key]), key
    gm.close()


def test_batch_empty_map_and_nothing_visible():
    """A map with no triangles, and one whose only triangles are behind the camera: the
    persistent kernel still runs every phase (and every LM iteration) and reports zero cost."""
    cam = cases.small_pinhole()
    intr = rm.Intrinsics.from_camera(cam)
    depth = np.full((cam.height, cam.width), 2.0, np.float32)
    cls = np.zeros((cam.height, cam.width), np.uint8)
    scan = rm.Scan.make(intr, depth, cls)
    v, f = cases.plane_grid(3, 3, (-1, -1, -2.0), (2, 0, 0), (0, 2, 0))
    for mesh in ((np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32)), (v, f)):
        gm = rm.Map(mesh[0], mesh[1], np.zeros(len(mesh[1]), np.uint8))
        b = rm.cost_grad_batch(gm, [(scan, np.eye(4))] * 3)
        assert int(b["counts"].sum()) == 0 and float(b["e_ls"].abs().sum()) == 0.0
        poses, reps, status = rm.align_batch(gm, [(scan, np.eye(4))] * 2, max_iters=3)
        assert status in ("RM_OK", "RM_ENOTCONV")
        assert np.allclose(poses, np.eye(4)[None])
        gm.close()


def test_batch_icp_equals_single_calls(mixed):
    """ICP alignment of the mixed batch in one persistent launch: every problem's pose and
    report equal its rm_icp_align call bit for bit, and the Lidar problems end near the truth."""
    gm = mixed["gm"]
    gm.set_tuning()
    probs = mixed["probs"]
    poses, reps, status = rm.icp_align_batch(gm, [(pr["gscan"], pr["start"]) for pr in probs], tol=0.5,
                                             max_iters=8, step_tol=1e-4)
    for k, pr in enumerate(probs):
        ps, rs = rm.icp_align(gm, pr["gscan"], pr["start"], tol=0.5, max_iters=8, step_tol=1e-4)
        assert np.array_equal(poses[k], ps), k
        for f in ("iters", "converged", "n_assoc", "cost_l1_initial", "cost_l1_final"):
            assert reps[k][f] == rs[f], (k, f, reps[k][f], rs[f])
    for k, pr in enumerate(probs):
        if pr["cam"].model == "spherical":
            assert reps[k]["converged"] == 1
            assert np.linalg.norm(poses[k][:3, 3] - pr["gt"][:3, 3]) < 0.02
    # repeated call (replayed graph) gives the same poses
    poses2, _, _ = rm.icp_align_batch(gm, [(pr["gscan"], pr["start"]) for pr in probs], tol=0.5,
                                      max_iters=8, step_tol=1e-4)
    assert np.array_equal(poses, poses2)
