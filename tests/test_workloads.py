"""The seeded generators: C and numpy agree, and the scenes have the structure they claim."""
import numpy as np

import workloads as W


def test_rng_c_matches_numpy():
    lib = W._L()
    for seed, stream in ((0, 0), (1, 2), (12345, 2000007), (2**63 + 5, 9)):
        idx = np.array([0, 1, 2, 1000, 2**40 + 3], dtype=np.uint64)
        ref = [lib.wl_rng(seed, stream, int(i)) for i in idx]
        assert [int(v) for v in W.rng(seed, stream, idx)] == ref


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 0 (base = mix(0) = 0 when seed=0, stream=0): the first outputs of the
    # published generator with state 0 are 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F.
    base_zero = W.rng(0, 0, np.array([0, 1, 2], dtype=np.uint64))
    assert W._mix64(np.array([0], dtype=np.uint64))[0] == 0
    assert [hex(int(v)) for v in base_zero] == ["0xe220a8397b1dcdaf", "0x6e789e6aa1b965f4", "0x6c45d188009454f"]


def test_bernoulli_rate_and_match():
    n = 1 << 20
    a = W.bernoulli(3, 0, 0.02, n)
    thr = np.uint64(W.bernoulli_threshold(0.02))
    b = (W.rng(3, 0, np.arange(n, dtype=np.uint64)) < thr).astype(np.uint8)
    assert np.array_equal(a, b)
    assert abs(a.mean() - 0.02) < 0.001


def test_tunnel_walls_are_shells():
    dims = (128, 128, 64)
    occ = W.tunnel_scene(2, dims, ntunnels=4, rmin=6, rmax=10)
    radii, lines = W.tunnel_lines(2, dims, ntunnels=4, rmin=6, rmax=10)
    z, y, x = np.nonzero(occ)
    pts = np.stack([x, y, z], 1).astype(np.float64)[::13]
    # distance of each wall voxel to each tunnel's polyline
    inside_any = np.zeros(len(pts), bool)
    on_shell = np.zeros(len(pts), bool)
    for r, line in zip(radii, lines):
        a, b = line[:-1], line[1:]
        u = b - a
        w = pts[:, None, :] - a[None]
        t = np.clip((w * u[None]).sum(-1) / np.maximum((u * u).sum(-1), 1e-300)[None], 0, 1)
        d2 = ((w - t[..., None] * u[None]) ** 2).sum(-1).min(1)
        inside_any |= d2 < r * r
        on_shell |= (d2 >= r * r) & (d2 < (r + 1.5) ** 2)
    assert on_shell.all() and not inside_any.any()


def test_lidar_deterministic_and_sized():
    dims = (96, 96, 48)
    truth = W.tunnel_scene(4, dims, ntunnels=3, rmin=5, rmax=8)
    _, lines = W.tunnel_lines(4, dims, ntunnels=3, rmin=5, rmax=8)
    out = []
    for threads in (1, 3):
        seq = W.LidarSequence(truth, 4, lines[0], nframes=4, nbeams=8, nazim=64, maxrange=60, threads=threads)
        out.append([seq.next() for _ in range(3)])
    for (xa, va), (xb, vb) in zip(*out):
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    xyz, val = out[0][0]
    assert len(val) > 0 and (val == 1).sum() > 0
    assert (xyz >= 0).all() and (xyz[:, 0] < 96).all() and (xyz[:, 2] < 48).all()


def test_batched_params_ranges():
    sides = []
    for m in range(96):
        s, p, nb = W.batched_params(7, m)
        assert s % 8 == 0 and 32 <= s <= 512 and 0.01 <= p <= 0.05 and 0 <= nb <= 20
        sides.append(s)
    assert min(sides) < 64 and max(sides) > 256
    g = W.batched_map(7, int(np.argmin(sides)))
    assert g.shape == (min(sides),) * 3 and 0 < g.mean() < 0.6


def test_free_points_are_free():
    occ = W.bernoulli_grid(1, (20, 21, 22), 0.2)
    pts = W.free_points(5, occ, 0.1, 2000)
    v = np.clip(np.floor(pts.astype(np.float64) / 0.1 + 0.5).astype(int), 0, [21, 20, 19])
    assert (occ[v[:, 2], v[:, 1], v[:, 0]] == 0).mean() > 0.999
