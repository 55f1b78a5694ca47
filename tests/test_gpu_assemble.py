"""GPU parity: contact assembly is bit-exact with the oracle (Sec. 2.2, 3.3)."""
import numpy as np
import pytest
import torch

from gpu_common import Problem, to_np
from paper_1808_02558_gb300 import binding, workload
from synth import Scene, box_scene, lattice_scene, scene_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding.Context()


def check_bitexact(pb: Problem):
    con, o = pb.con, pb.oc
    assert con.Nc == o.Nc and con.M == pb.scene.M and con.P == pb.P and con.L == pb.L
    if o.Nc == 0:
        return
    a = to_np(workload.view(con, "body_a"))
    b = to_np(workload.view(con, "body_b"))
    assert np.array_equal(a, o.a) and np.array_equal(b, o.b)
    assert np.array_equal(to_np(workload.view(con, "plane")), o.plane)
    key = to_np(workload.view(con, "key")).view(np.uint64)
    assert np.array_equal(key, o.key)
    assert np.array_equal(to_np(workload.view(con, "phi")), o.phi)
    F = to_np(workload.view(con, "frame")).reshape(9, -1)
    assert np.array_equal(F[0:3].T, o.n) and np.array_equal(F[3:6].T, o.t1) and np.array_equal(F[6:9].T, o.t2)
    assert np.array_equal(to_np(workload.view(con, "point")).reshape(3, -1).T, o.p)
    assert np.array_equal(to_np(workload.view(con, "arm_b")).reshape(3, -1).T, o.rb)
    assert np.array_equal(to_np(workload.view(con, "arm_a")).reshape(3, -1).T, o.ra)
    r = to_np(workload.view(con, "r"))
    want = pb.pad(pb.r)
    assert np.abs(r - want).max() <= 1e-12 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("name,seed", [("pile8", 1), ("pile8", 2), ("pile8", 3), ("pile20", 1), ("pile40p", 1)])
def test_assemble_configs_bitexact(ctx, name, seed):
    check_bitexact(Problem(ctx, scene_for(name, seed)))


@pytest.mark.parametrize("slots", [3, 4])
def test_assemble_polydisperse_small(ctx, slots):
    check_bitexact(Problem(ctx, lattice_scene(7, 5, polydisperse=True), slots))


def test_assemble_edge_cases(ctx):
    z = np.zeros((1, 3))
    # one sphere above the floor: no contact at all
    one = Scene(name="free", pos=[[0.0, 0.0, 3.0]], vel=z, omega=z, radius=[0.5])
    check_bitexact(Problem(ctx, one))
    # one sphere on the floor: one contact, 3 rows padded to 4
    check_bitexact(Problem(ctx, Scene(name="sop", pos=[[0.2, 0.1, 0.49]], vel=[[0.1, 0, 0]], omega=z, radius=[0.5])))
    # two coincident-in-x spheres stacked: ties in the tangent choice
    two = Scene(name="stack", pos=[[0.0, 0.0, 0.5], [0.0, 0.0, 1.45]], vel=np.zeros((2, 3)),
                omega=np.zeros((2, 3)), radius=[0.5, 0.5])
    check_bitexact(Problem(ctx, two))
    # ragged lattice (not a power of two) with a large envelope
    check_bitexact(Problem(ctx, lattice_scene(5, 9, polydisperse=True, delta=0.45)))


def test_assemble_walled_box_small(ctx):
    # 6 x 6 x 3 box: spheres against both walls of each side axis, in the
    # corners against two walls and the floor at once (ties ordered by plane)
    check_bitexact(Problem(ctx, box_scene(1, n=6, layers=3)))
    check_bitexact(Problem(ctx, box_scene(2, n=5, layers=2, lift=1.0), 4))


def test_assemble_walled_box_full(ctx):
    # 64 000 spheres in the 40 x 40 x 80 box
    pb = Problem(ctx, scene_for("box40", 1))
    check_bitexact(pb)
    a, b = to_np(workload.view(pb.con, "body_a")), to_np(workload.view(pb.con, "body_b"))
    planes = a == pb.scene.M
    # floor contacts have normal +e_z, wall contacts normal +-e_x or +-e_y
    n = to_np(workload.view(pb.con, "frame")).reshape(9, -1)[0:3].T[planes]
    assert np.all(np.abs(n).max(axis=1) == 1.0)
    assert (np.abs(n[:, 0]) == 1.0).sum() > 0 and (np.abs(n[:, 1]) == 1.0).sum() > 0


def test_assemble_wall_arguments(ctx):
    s = box_scene(1, n=3, layers=1)
    c = binding.Context()
    dev = workload.scene_to_device(s, "cuda")
    for walls in [((0, 1, 0.0),) * 5, ((3, 1, 0.0),), ((0, 0, 0.0),), ((1, 2, 0.0),)]:
        with pytest.raises(binding.QPError) as e:
            c.assemble(dev, s.floor_z, s.gravity, s.dt, s.delta, s.mu, 3, walls)
        assert e.value.code == binding.QP_INVALID_ARG
    c.close()
