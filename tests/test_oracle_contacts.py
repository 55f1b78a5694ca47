"""Oracle pins for contact detection, frames and ordering (Sec. 2.2, 3.3)."""
import numpy as np

from oracle import contacts as oc
from synth import Scene, lattice_scene


def test_pairs_match_bruteforce_polydisperse():
    s = lattice_scene(5, 7, polydisperse=True)
    fast = oc._pairs_within(s.pos, s.radius, s.delta)
    slow = oc.candidate_pairs_bruteforce(s.pos, s.radius, s.delta)
    assert np.array_equal(fast, slow)


def test_pairs_match_bruteforce_random_cloud():
    rng = np.random.default_rng(3)
    pos = rng.uniform(0, 4, size=(150, 3))
    rad = rng.uniform(0.2, 0.5, size=150)
    fast = oc._pairs_within(pos, rad, 0.05)
    slow = oc.candidate_pairs_bruteforce(pos, rad, 0.05)
    assert np.array_equal(fast, slow)


def test_lattice_contact_count_is_face_pairs_plus_floor():
    # every face-neighbour pair overlaps (spacing 0.98 < diameter) and the
    # bottom layer touches the floor: 3 n^2 (n-1) + n^2 contacts, all face pairs
    for n in (3, 8):
        s = lattice_scene(n, 1)
        c = oc.detect(s)
        assert c.Nc == 3 * n * n * (n - 1) + n * n
        pair = c.a < s.M
        da = np.abs(np.array(np.unravel_index(c.a[pair], (n, n, n))) -
                    np.array(np.unravel_index(c.b[pair], (n, n, n))))
        assert np.all(da.sum(axis=0) == 1)
        assert np.sum(~pair) == n * n


def test_two_sphere_geometry_by_hand():
    s = Scene(name="two", pos=[[0.0, 0.0, 5.0], [0.9, 0.0, 5.0]], vel=np.zeros((2, 3)),
              omega=np.zeros((2, 3)), radius=[0.5, 0.5])
    c = oc.detect(s)
    assert c.Nc == 1 and c.a[0] == 0 and c.b[0] == 1
    assert c.phi[0] == 0.9 - 1.0
    assert np.array_equal(c.n[0], [1.0, 0.0, 0.0])
    # p = x_a + n (r_a + phi/2) = 0.5 + (-0.1)/2 = 0.45
    assert np.allclose(c.p[0], [0.45, 0.0, 5.0], rtol=0, atol=1e-15)
    # e = y (lowest index among |n_y| = |n_z| = 0): t1 = n x e_y = (0, 0, 1), t2 = n x t1 = (0, -1, 0)
    assert np.array_equal(c.t1[0], [0.0, 0.0, 1.0])
    assert np.array_equal(c.t2[0], [0.0, -1.0, 0.0])
    assert np.allclose(c.ra[0], [0.45, 0, 0]) and np.allclose(c.rb[0], [-0.45, 0, 0])


def test_floor_contact_geometry_by_hand():
    s = Scene(name="one", pos=[[1.0, 2.0, 0.48]], vel=np.zeros((1, 3)), omega=np.zeros((1, 3)), radius=[0.5])
    c = oc.detect(s)
    assert c.Nc == 1 and c.a[0] == 1 and c.b[0] == 0  # static floor is body M = 1
    assert np.isclose(c.phi[0], -0.02, atol=1e-15)
    assert np.array_equal(c.n[0], [0.0, 0.0, 1.0])
    assert np.allclose(c.p[0], [1.0, 2.0, -0.01], atol=1e-15)
    assert np.allclose(c.rb[0], [0.0, 0.0, -0.49], atol=1e-15)
    frame = np.stack([c.n[0], c.t1[0], c.t2[0]])
    assert np.allclose(frame @ frame.T, np.eye(3), atol=1e-15)


def test_frames_orthonormal_right_handed():
    s = lattice_scene(4, 2, polydisperse=True)
    c = oc.detect(s)
    F = np.stack([c.n, c.t1, c.t2], axis=1)
    assert np.allclose(np.einsum("cij,ckj->cik", F, F), np.eye(3), atol=1e-14)
    assert np.allclose(np.linalg.det(F), 1.0, atol=1e-14)


def test_morton_interleave_known_bits():
    one = np.array([1])
    zero = np.array([0])
    assert oc.morton_interleave(one, zero, zero)[0] == 1
    assert oc.morton_interleave(zero, one, zero)[0] == 2
    assert oc.morton_interleave(zero, zero, one)[0] == 4
    assert oc.morton_interleave(np.array([2]), zero, zero)[0] == 8
    full = np.array([(1 << 21) - 1])
    assert oc.morton_interleave(full, full, full)[0] == (1 << 63) - 1
    assert oc.morton_interleave(np.array([5]), np.array([3]), np.array([6]))[0] == 0b101110011


def test_order_is_key_then_bodies():
    s = lattice_scene(6, 4, polydisperse=True)
    c = oc.detect(s)
    trip = list(zip(c.key.tolist(), c.a.tolist(), c.b.tolist()))
    assert trip == sorted(trip)
    assert len(set(zip(c.a.tolist(), c.b.tolist()))) == c.Nc


def test_wall_contacts_hand_computed():
    """One sphere against each side wall (an extension of the floor rule): gap
    sign (x_axis - offset) - r, normal sign e_axis into the box, contact point
    offset + sign Phi/2 on that axis, arm of the static wall zero."""
    from synth import Scene

    walls = ((0, 1, -1.0), (0, -1, 4.0), (1, 1, 0.0), (1, -1, 2.5))
    pos = np.array([[-0.55, 1.0, 3.0], [3.6, 1.0, 3.0], [1.5, 0.38, 3.0], [1.5, 2.05, 3.0]])
    rad = np.array([0.5, 0.45, 0.4, 0.5])
    s = Scene(name="walls", pos=pos, vel=np.zeros((4, 3)), omega=np.zeros((4, 3)), radius=rad, delta=0.05,
              walls=walls)
    c = oc.detect(s)
    assert c.Nc == 4 and np.all(c.a == 4)
    # plane index of each contact: 1 + the wall's position in the list
    assert sorted(zip(c.b.tolist(), c.plane.tolist())) == [(0, 1), (1, 2), (2, 3), (3, 4)]
    # the midpoint between the sphere surface and the wall
    want = {0: (-0.05, [1, 0, 0], [-1.025, 1.0, 3.0]), 1: (-0.05, [-1, 0, 0], [4.025, 1.0, 3.0]),
            2: (-0.02, [0, 1, 0], [1.5, -0.01, 3.0]), 3: (-0.05, [0, -1, 0], [1.5, 2.525, 3.0])}
    for k in range(4):
        b = int(c.b[k])
        phi, n, p = want[b]
        assert abs(c.phi[k] - phi) < 1e-12
        assert np.allclose(c.n[k], n) and np.allclose(c.p[k], p, atol=1e-12)
        assert np.all(c.ra[k] == 0.0)
        assert np.allclose(c.rb[k], np.array(p) - pos[b], atol=1e-12)
        assert abs(np.dot(c.t1[k], c.n[k])) < 1e-15 and abs(np.dot(c.t2[k], c.n[k])) < 1e-15
    # a sphere out of reach of every wall has no contact
    s2 = Scene(name="free", pos=np.array([[1.5, 1.2, 3.0]]), vel=np.zeros((1, 3)), omega=np.zeros((1, 3)),
               radius=np.array([0.5]), delta=0.05, walls=walls)
    assert oc.detect(s2).Nc == 0


def test_box_scene_counts_and_order():
    """Box scene: the floor under every bottom sphere and one wall contact per
    outer sphere and side; the order is total ((key, a, b) with the plane index
    breaking ties) and every pair is found by the brute-force search."""
    from synth import box_scene

    s = box_scene(1, n=6, layers=4)
    c = oc.detect(s)
    stat = c.a == s.M
    n, layers = 6, 4
    # the floor under the lower half of the checkerboard of the bottom layer
    assert int(stat.sum()) == n * n // 2 + 4 * n * layers
    floor = stat & (c.n[:, 2] == 1.0)
    assert int(floor.sum()) == n * n // 2
    pairs = oc.candidate_pairs_bruteforce(s.pos, s.radius, s.delta)
    assert int((~stat).sum()) == len(pairs)
    assert np.all(np.diff(c.key.astype(np.float64)) >= 0)


def test_box40_starts_without_overlap():
    """The 64 000-sphere box starts with every gap (pairs, floor, walls) >= 0:
    the spheres fall, nothing is pushed apart by an initial overlap."""
    from synth import scene_for

    s = scene_for("box40", 1)
    c = oc.detect(s)
    assert s.M == 64000 and c.Nc > 50000
    assert c.phi.min() >= 0.0
    side = s.walls[1][2]
    assert side == 40.0 and s.pos[:, 2].max() < 2.0 * side
