"""GPU parity of closestPoint / adjacentHyperplane (plan_obstacle_planes)
against the FP64 oracle (oracle/planes.py).

Bar: FP32 arithmetic on FP32-rounded inputs.  Closest points and distances
within 2e-5 x (1 + the coordinate scale) of the oracle (the faces and edge
segments come rounded from FP64 and each candidate costs a dozen FP32
operations, so the error is a small multiple of 2^-24 times the scale,
whatever the angle at a vertex); the plane's unit normal within 1e-4 of the
oracle's, its offset within the point tolerance plus 1e-4 m |z|, and the
plane through the closest point at the distance from the point, wherever the
distance exceeds 1e-3; the nearest obstacle exact unless its distance is within the
tolerance of the runner-up (then the distances are compared)."""
import numpy as np
import pytest

from oracle import planes as OP
from paper_2411_13507_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # the -m gpu run happens on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2411_13507_gb300 import plan as P  # noqa: E402


def planner(m):
    bounds = (2.0, 4.0) if m == 2 else (3.0, 6.0, 30.0)
    return P.Planner(m, m, 5, bounds, arith="f32", input="f32")


def run(m, points, obs, nearest_only=False):
    pl = planner(m)
    pts = torch.as_tensor(np.asarray(points, dtype=np.float32)).cuda()
    do = P.obstacles_to_device(obs, input="f32")
    out = pl.obstacle_planes(pts, do, nearest_only=nearest_only)
    return {k: v.cpu().numpy() for k, v in out.items()}, pl.info()


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def compare(points, obs, gpu, rows=None):
    pts = f32(points)
    A, b = f32(obs.A), f32(obs.b)
    rows = range(pts.shape[0]) if rows is None else rows
    orc = OP.planes(pts[list(rows)], obs.off, A, b)
    scale = 1.0 + max(np.abs(pts).max(), np.abs(b).max())
    tol = 2e-5 * scale
    m = pts.shape[1]
    for k, p in enumerate(rows):
        dz = np.abs(gpu["closest"][p] - orc["closest"][k]).max()
        assert dz <= tol, (p, dz)
        assert np.abs(gpu["dist"][p] - orc["dist"][k]).max() <= tol
        far = orc["dist"][k] > 1e-3
        assert np.abs(gpu["plane"][p][far, :m] - orc["plane"][k][far, :m]).max(initial=0) <= 1e-4
        # the offset l = h . z carries the normal's error times |z|; the plane
        # itself must pass through z and lie at distance d from the point
        zmax = np.abs(orc["closest"][k][far]).max(initial=0.0)
        assert np.abs(gpu["plane"][p][far, m] - orc["plane"][k][far, m]).max(initial=0) <= tol + 1e-4 * m * zmax
        hg, lg = gpu["plane"][p][far, :m].astype(np.float64), gpu["plane"][p][far, m].astype(np.float64)
        zg = gpu["closest"][p][far].astype(np.float64)
        assert np.abs(np.sum(hg * zg, axis=1) - lg).max(initial=0) <= tol
        assert np.abs(hg @ pts[p] - lg - gpu["dist"][p][far]).max(initial=0) <= tol
        inside = orc["dist"][k] == 0.0
        assert np.all(gpu["dist"][p][inside] == 0.0) and np.all(gpu["plane"][p][inside] == 0.0)
        # nearest obstacle
        d = np.sort(orc["dist"][k])
        if gpu["nearest"][p] != orc["nearest"][k]:
            assert len(d) > 1 and d[1] - d[0] <= tol
        assert abs(gpu["nearest_dist"][p] - orc["nearest_dist"][k]) <= tol
    return orc


@pytest.mark.parametrize("seed", [1, 2])
def test_planes_2d_all_pairs(seed):
    prob, obs = synth.keepout_2d(seed, N=300, n_obst=40, dtype="f32")
    pts = prob.states[:, :2]
    gpu, info = run(2, pts, obs)
    compare(pts, obs, gpu)


@pytest.mark.parametrize("seed", [1, 2])
def test_planes_3d_all_pairs(seed):
    rng = np.random.default_rng(seed)
    obs = synth.obstacles(seed, 30, 3, (0.0, 10.0), (0.5, 2.0), 3, dtype="f32")
    pts = rng.uniform(0.0, 10.0, size=(200, 3))
    gpu, info = run(3, pts, obs)
    compare(pts, obs, gpu)


def test_planes_full_size_sampled_points():
    """5000 nodes x 500 obstacles (2.5 M pairs) on the GPU; every 50th node
    against the oracle."""
    prob, obs = synth.keepout_2d(1, dtype="f32")
    pts = prob.states[:, :2]
    gpu, info = run(2, pts, obs)
    compare(pts, obs, gpu, rows=range(0, prob.N, 50))
    # the nearest-only mode prunes pairs by distance bounds: same nearest
    # obstacle and distance bits as the all-pairs mode, for every node
    near, _ = run(2, pts, obs, nearest_only=True)
    assert np.array_equal(near["nearest"], gpu["nearest"])
    assert np.array_equal(near["nearest_dist"], gpu["nearest_dist"])


def test_points_inside_sixteen_row_obstacles_and_nearest_only():
    th = 2 * np.pi * (np.arange(16) + 0.5) / 16
    nrm = np.stack([np.cos(th), np.sin(th)], axis=1)
    centers = np.array([[1.0, 1.0], [3.0, 1.5], [2.0, 3.0]])
    A = np.tile(nrm, (3, 1))
    b = np.concatenate([nrm @ c + 0.4 for c in centers])
    obs = synth.Obstacles(np.array([0, 16, 32, 48], dtype=np.int32), A, b)
    rng = np.random.default_rng(3)
    pts = np.concatenate([centers + rng.uniform(-0.1, 0.1, size=centers.shape), rng.uniform(0, 4, size=(60, 2))])
    gpu, info = run(2, pts, obs)
    compare(pts, obs, gpu)
    assert np.all(gpu["dist"][np.arange(3), np.arange(3)] == 0.0)
    near, _ = run(2, pts, obs, nearest_only=True)
    assert np.array_equal(near["nearest"], gpu["nearest"]) and np.array_equal(near["nearest_dist"], gpu["nearest_dist"])


def test_no_obstacles():
    obs = synth.Obstacles(np.zeros(1, dtype=np.int32), np.zeros((0, 2)), np.zeros(0))
    gpu, info = run(2, np.ones((5, 2)), obs, nearest_only=True)
    assert np.all(gpu["nearest"] == -1) and np.all(np.isinf(gpu["nearest_dist"]))
