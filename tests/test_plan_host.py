"""Host setup (no GPU): the C ABI surface, hierarchy invariants of Sec. 4.5,
Alg. 3 colouring and symbolic Galerkin patterns against the oracle, the
Dirichlet reduction, error statuses and plan save/load."""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth
import paper_2104_13755_gb300 as smg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "smg.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = sorted(set(re.findall(r"\b(smg_[a-z0-9_]+)\s*\(", hdr)))
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(smg.lib, n)]
    assert not missing, missing


@pytest.fixture(scope="module")
def ico_plan():
    V, F = synth.perturbed_icosphere(4, seed=0)
    return V, F, smg.Plan(V, F, max_levels=3, min_coarse=0)


@pytest.fixture(scope="module")
def disk_plan():
    V, F, bnd = synth.disk(60, seed=3)
    return V, F, bnd, smg.Plan(V, F, dirichlet=bnd, min_coarse=100)


def test_level_sizes_follow_ratio_rule(ico_plan):
    V, F, p = ico_plan
    assert [p.level_info(l)[0] for l in range(p.num_levels)] == [2562, 640, 160]
    V2, F2 = synth.torus(80, 40)
    p2 = smg.Plan(V2, F2)                        # paper default: coarsest >= 500
    sizes = [p2.level_info(l)[0] for l in range(p2.num_levels)]
    assert sizes == [3200, 800]
    p3 = smg.Plan(V2, F2, max_coarse=300)       # coarsen while n > 300
    sizes3 = [p3.level_info(l)[0] for l in range(p3.num_levels)]
    assert sizes3 == [3200, 800, 200]


def test_prolongation_rows_are_barycentric(ico_plan, disk_plan):
    for plan in (ico_plan[2], disk_plan[3]):
        for l in range(1, plan.num_levels):
            idx, w, nc = plan.prolongation(l)
            used = idx >= 0
            assert np.all(w[used] > 0) and np.all(w[~used] == 0)
            assert np.abs(w.sum(1) - 1.0).max() < 1e-14
            assert np.all(used.sum(1) >= 1) and idx.max() < nc
            P = plan.prolongation_csr(l)
            assert np.abs(P @ np.ones(nc) - 1).max() < 1e-14        # P reproduces constants
            assert np.all(np.asarray((P != 0).sum(0)).ravel() >= 1)  # full column support


def test_levels_keep_topology(ico_plan, disk_plan):
    for plan, chi in ((ico_plan[2], 2), (disk_plan[3], 1)):
        for l in range(plan.num_levels):
            V, F = plan.mesh(l)
            assert synth.euler_characteristic(V.shape[0], F) == chi
    V, F = synth.torus(60, 20)
    p = smg.Plan(V, F, min_coarse=50)
    for l in range(p.num_levels):
        Vl, Fl = p.mesh(l)
        assert synth.euler_characteristic(Vl.shape[0], Fl) == 0


def test_planar_interior_linear_reproduction():
    """On a planar mesh every interior collapse flattens both patches exactly (zero
    LSCM energy), so barycentric prolongation reproduces x and y away from the
    boundary, where boundary collapses snap UVs."""
    V, F, bnd = synth.disk(50, seed=5)
    p = smg.Plan(V, F, max_levels=2, min_coarse=0)
    Vc, _ = p.mesh(1)
    P = p.prolongation_csr(1)
    r = np.linalg.norm(V[:, :2], axis=1)
    inner = r < 0.6
    err = np.abs(P @ Vc[:, :2] - V[:, :2])[inner].max()
    assert err < 1e-10


def test_colouring_and_patterns_match_oracle(ico_plan, disk_plan):
    for case in (ico_plan, disk_plan):
        V, F, plan = case[0], case[1], case[-1]
        known = case[2] if len(case) == 4 else np.zeros(V.shape[0], dtype=bool)
        A = oracle.system_matrix(V, F, 1e-3)
        Ps = [plan.prolongation_csr(l) for l in range(1, plan.num_levels)]
        A, Ps, u, keep = oracle.dirichlet_reduce(A, Ps, known)
        assert np.array_equal(plan.unknowns(), u)
        if keep is not None:
            assert np.array_equal(plan.kept_coarse(), keep)
        S = A
        for l in range(plan.num_levels):
            rp, ci = plan.pattern(l)
            Sp = S.tocsr()
            Sp.sort_indices()
            assert np.array_equal(rp, Sp.indptr) and np.array_equal(ci, Sp.indices)
            if l < plan.num_levels - 1:
                col = plan.colouring(l)
                assert np.array_equal(col, oracle.greedy_colouring(Sp))   # bit-exact
                S = oracle.galerkin_pattern(Sp, Ps[l])


def test_invalid_meshes_report_status():
    V, F = synth.icosphere(1)
    bad = F.copy()
    bad[0, 0] = 1000
    with pytest.raises(smg.SmgError) as e:
        smg.Plan(V, bad)
    assert e.value.status == 1
    flipped = F.copy()
    flipped[0] = flipped[0, [0, 2, 1]]
    with pytest.raises(smg.SmgError) as e:
        smg.Plan(V, flipped)
    assert e.value.status == 2
    with pytest.raises(smg.SmgError) as e:
        smg.Plan(V, F, dirichlet=np.ones(V.shape[0], dtype=bool))
    assert e.value.status == 1


def test_plan_save_load_roundtrip(tmp_path, disk_plan):
    plan = disk_plan[3]
    path = str(tmp_path / "disk.smgplan")
    plan.save(path)
    q = smg.Plan.load(path)
    assert q.num_levels == plan.num_levels
    for l in range(plan.num_levels):
        assert q.level_info(l) == plan.level_info(l)
        for a, b in zip(q.pattern(l), plan.pattern(l)):
            assert np.array_equal(a, b)
        if l >= 1:
            assert np.array_equal(q.prolongation(l)[1], plan.prolongation(l)[1])
    with open(path, "r+b") as f:
        f.write(b"XXXX")
    with pytest.raises(smg.SmgError) as e:
        smg.Plan.load(path)
    assert e.value.status == 11


def test_plan_is_bitwise_deterministic(tmp_path):
    """Setup is deterministic: two builds of the same mesh save identical
    bytes.  The mesh is large enough (> 4096 rows at level 0) that the
    Galerkin and transfer plans are built on several host threads."""
    V, F = synth.perturbed_icosphere(5, seed=2)
    blobs = []
    for k in range(2):
        path = str(tmp_path / ("p%d.smgplan" % k))
        smg.Plan(V, F).save(path)
        with open(path, "rb") as f:
            blobs.append(f.read())
    assert len(blobs[0]) > 0 and blobs[0] == blobs[1]


@pytest.mark.parametrize("dirichlet", [False, True])
def test_two_ring_plan_patterns_and_colouring_match_oracle(dirichlet):
    """pattern_rings = 2 (Sec. 6: Bilaplacian-type systems): the level-0 pattern
    is the oracle's 2-ring pattern restricted to the unknowns, every coarse
    pattern its Galerkin pattern, and every colouring the oracle's Alg. 3."""
    if dirichlet:
        V, F, known = synth.disk(24, seed=3)
    else:
        V, F = synth.torus(40, 16, seed=1)
        known = np.zeros(V.shape[0], dtype=bool)
    plan = smg.Plan(V, F, dirichlet=known if dirichlet else None, pattern_rings=2, min_coarse=60)
    A = oracle.bilaplacian_system(V, F, 1e-3)
    Ps = [plan.prolongation_csr(l) for l in range(1, plan.num_levels)]
    A, Ps, u, _ = oracle.dirichlet_reduce(A, Ps, known)
    S = A
    for l in range(plan.num_levels):
        rp, ci = plan.pattern(l)
        Sp = S.tocsr()
        Sp.sort_indices()
        assert np.array_equal(rp, Sp.indptr) and np.array_equal(ci, Sp.indices), l
        if l < plan.num_levels - 1:
            assert np.array_equal(plan.colouring(l), oracle.greedy_colouring(Sp))
            S = oracle.galerkin_pattern(Sp, Ps[l])


@pytest.mark.parametrize("dirichlet", [False, True])
def test_block3_plan_patterns_and_colouring_match_oracle(dirichlet):
    """block_size = 3 (3|V| systems, Sec. 6): level 0 is the vertex pattern in
    3 x 3 blocks over the unknowns, P is P (x) I_3, every coarse pattern follows
    from them as for scalar systems, and every colouring is Alg. 3 on the
    vertex pattern with the components in order (oracle.block_colouring)."""
    if dirichlet:
        V, F, known = synth.disk(20, seed=2)
    else:
        V, F = synth.perturbed_icosphere(3, seed=1)
        known = np.zeros(V.shape[0], dtype=bool)
    plan = smg.Plan(V, F, dirichlet=known if dirichlet else None, block_size=3, min_coarse=60)
    A = oracle.expand_blocks(oracle.system_matrix(V, F, 1e-3), 3)
    A = oracle.on_pattern(oracle.block_pattern(oracle.mesh_pattern(V.shape[0], F), 3), A)
    Ps = [oracle.expand_blocks(plan.prolongation_csr(l), 3) for l in range(1, plan.num_levels)]
    A, Ps, u, _ = oracle.dirichlet_reduce(A, Ps, np.repeat(known, 3))
    assert plan.level_info(0)[0] == u.size
    S = A
    for l in range(plan.num_levels):
        rp, ci = plan.pattern(l)
        Sp = S.tocsr()
        Sp.sort_indices()
        assert np.array_equal(rp, Sp.indptr) and np.array_equal(ci, Sp.indices), l
        if l < plan.num_levels - 1:
            assert np.array_equal(plan.colouring(l), oracle.block_colouring(Sp, 3))
            S = oracle.galerkin_pattern(Sp, Ps[l])
