"""Derivative-free alignment on the Table I cost (Sec. IV.C) on the GPU vs the CPU oracle,
through the C ABI: Nelder-Mead or Powell's method, then coordinate descent.

Table I counts are bit-exact between the two sides and both take the search's decisions on
those integers with the same rules, so the two searches follow the same path: the same number
of scored poses, iterations and shrinks, the same final cost, and final poses that differ only
by the rounding of the SE(3) exponential.
"""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import cases
import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker is deselected on CPU
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1702_06813_gb300 as rm  # noqa: E402
from paper_1702_06813_gb300 import build as rmbuild  # noqa: E402

rmbuild.build()


def _gap(P, Q):
    return (float(np.linalg.norm(P[:3, 3] - Q[:3, 3])),
            math.degrees(Rotation.from_matrix(P[:3, :3].T @ Q[:3, :3]).magnitude()))


def _same_search(g, grep, o, orep):
    for key in ("evals", "nm_iters", "nm_shrinks", "cd_iters", "converged", "powell_iters"):
        assert grep[key] == orep[key], (key, grep, orep)
    assert grep["e_table_final"] == orep["e_table"], (grep, orep)
    dt, da = _gap(g, o)
    assert dt < 1e-9 and da < 1e-7, (dt, da)


@pytest.mark.parametrize("noise", [0.0, 0.01])
def test_dfo_matches_oracle_pinhole(noise):
    c = cases.config1(seed=1900, noise=0.0, dropout=0.0)
    mesh, cam = c["mesh"], c["cam"]
    gt = synth.pose_from(c["gt"][:3, 3], 0.7, math.radians(25.0), 0.0)
    start = synth.perturb_fixed(gt, cases.rng(4), 0.03, 1.5)
    sd, sc = synth.synth_scan(mesh, cam, gt, cases.rng(6), sigma_abs=noise)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(cam), sd, sc)
    d = rm.dfo_params(nm_iters=150, cd_iters=80)
    od = oracle.dfo_params(nm_iters=150, cd_iters=80)
    pg, rep = rm.dfo_align(gm, scan, start, dfo=d)
    po, orep = om.dfo_align(start, cam, sd, sc, dfo=od)
    _same_search(pg, rep, po, orep)
    assert rep["e_table_initial"] == om.cost(start, cam, sd, sc)["e_table"]
    assert rep["e_table_final"] == om.cost(pg, cam, sd, sc)["e_table"]
    assert rep["e_table_final"] < rep["e_table_initial"]
    gm.close()


def test_dfo_matches_oracle_raytable():
    w = synth.workload_lidar(seed=4300, target_fo=100_000, target_fu=40_000, n_panels=60)
    mesh, cam = w["mesh"], w["cam"]
    sd, sc = w["scan"]
    start = synth.perturb_fixed(w["gt"], cases.rng(7), 0.1, 1.0)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(cam), sd, sc)
    d = rm.dfo_params(nm_iters=60, cd_iters=30, scale_t=0.1, scale_r=0.02)
    od = oracle.dfo_params(nm_iters=60, cd_iters=30, scale_t=0.1, scale_r=0.02)
    pg, rep = rm.dfo_align(gm, scan, start, dfo=d)
    po, orep = om.dfo_align(start, cam, sd, sc, dfo=od)
    _same_search(pg, rep, po, orep)
    gm.close()


def test_dfo_edge_cases():
    c = cases.config1(seed=1910)
    mesh, cam = c["mesh"], c["cam"]
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(cam), *c["scan"])
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    # no iterations: the best vertex of the first simplex, not converged
    pg, rep = rm.dfo_align(gm, scan, c["start"], dfo=rm.dfo_params(nm_iters=0, cd_iters=0))
    po, orep = om.dfo_align(c["start"], cam, *c["scan"], dfo=oracle.dfo_params(nm_iters=0, cd_iters=0))
    assert rep["status"] == "RM_ENOTCONV" and rep["evals"] == 7
    _same_search(pg, rep, po, orep)
    # the hybrid: gradient steps first, then the search from where they ended
    ph, hrep = rm.dfo_align(gm, scan, c["start"], dfo=rm.dfo_params(nm_iters=40, cd_iters=40), gd_iters=5)
    assert "gd" in hrep and hrep["e_table_final"] <= hrep["e_table_initial"]
    with pytest.raises(rm.RenderMapError):
        rm.dfo_align(gm, scan, c["start"], dfo=rm.dfo_params(scale_t=0.0))
    # Powell with no iterations: the origin, then coordinate descent from it
    pg, rep = rm.dfo_align(gm, scan, c["start"], dfo=rm.dfo_params(method="powell", powell_iters=0, cd_iters=3))
    po, orep = om.dfo_align(c["start"], cam, *c["scan"],
                            dfo=oracle.dfo_params(method="powell", powell_iters=0, cd_iters=3))
    assert rep["evals"] == 1 + 12 * rep["cd_iters"]
    _same_search(pg, rep, po, orep)
    for bad in (dict(method="powell", powell_step=0.0), dict(method="powell", powell_iters=-1),
                dict(method="powell", powell_tol=-1.0)):
        with pytest.raises(rm.RenderMapError):
            rm.dfo_align(gm, scan, c["start"], dfo=rm.dfo_params(**bad))
    d = rm.dfo_params()
    d.method = 2
    with pytest.raises(rm.RenderMapError):
        rm.dfo_align(gm, scan, c["start"], dfo=d)
    gm.close()


@pytest.mark.parametrize("noise", [0.0, 0.01])
def test_powell_matches_oracle_pinhole(noise):
    """Powell's method (the paper names it beside Nelder-Mead) then coordinate descent: the
    same line searches, iterations and replaced directions as the oracle, so the same path."""
    c = cases.config1(seed=1900, noise=0.0, dropout=0.0)
    mesh, cam = c["mesh"], c["cam"]
    gt = synth.pose_from(c["gt"][:3, 3], 0.7, math.radians(25.0), 0.0)
    start = synth.perturb_fixed(gt, cases.rng(4), 0.03, 1.5)
    sd, sc = synth.synth_scan(mesh, cam, gt, cases.rng(6), sigma_abs=noise)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(cam), sd, sc)
    pg, rep = rm.dfo_align(gm, scan, start, dfo=rm.dfo_params(method="powell", powell_iters=20, cd_iters=60))
    po, orep = om.dfo_align(start, cam, sd, sc, dfo=oracle.dfo_params(method="powell", powell_iters=20,
                                                                      cd_iters=60))
    _same_search(pg, rep, po, orep)
    assert rep["powell_iters"] >= 1 and rep["nm_iters"] == 0
    assert rep["e_table_final"] == om.cost(pg, cam, sd, sc)["e_table"]
    assert rep["e_table_final"] < rep["e_table_initial"]
    gm.close()


def test_powell_matches_oracle_raytable():
    w = synth.workload_lidar(seed=4300, target_fo=100_000, target_fu=40_000, n_panels=60)
    mesh, cam = w["mesh"], w["cam"]
    sd, sc = w["scan"]
    start = synth.perturb_fixed(w["gt"], cases.rng(7), 0.1, 1.0)
    om = oracle.OracleMap(mesh.vertices, mesh.faces, mesh.labels)
    gm = rm.Map(mesh.vertices, mesh.faces, mesh.labels)
    scan = rm.Scan.make(rm.Intrinsics.from_camera(cam), sd, sc)
    kw = dict(method="powell", powell_iters=3, cd_iters=10, scale_t=0.1, scale_r=0.02)
    pg, rep = rm.dfo_align(gm, scan, start, dfo=rm.dfo_params(**kw))
    po, orep = om.dfo_align(start, cam, sd, sc, dfo=oracle.dfo_params(**kw))
    _same_search(pg, rep, po, orep)
    gm.close()
