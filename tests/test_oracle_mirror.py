"""Pins of the oracle's FP32 key-generation mirror (Sec. 4.2 key generation
and sorting, Alg. 2 GenerateKeys, Eq. 11): tile bins checked against
brute-force scans of the region {q <= tau}, key layout, sort and ranges."""
import numpy as np
import pytest

import oracle
from paper_2605_04509_gb300 import synth


def make_inputs(K, M, C, W, H, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    conic = synth.random_conics(K * M, seed, 0.6, 12.0).reshape(K, M, 3)
    tau = rng.uniform(0.0, 11.0, (K, M)).astype(np.float32)
    tau[rng.uniform(size=(K, M)) < 0.05] = -1.0  # culled (k, i)
    depth = rng.uniform(0.3, 50.0, (K, M)).astype(np.float32)
    base = np.stack([rng.uniform(-20, W + 20, (K, M)), rng.uniform(-20, H + 20, (K, M))], -1)
    shift = rng.normal(0, 6.0 * spread, (K, M, C, 2))
    means = (base[:, :, None, :] + shift).astype(np.float32)
    means[rng.uniform(size=(K, M, C)) < 0.05] = np.nan  # culled view
    return conic, tau, depth, means


def tiles_of(keys, vals, counts, bit_k):
    """{(k, i): [tile ids in emission order]} from emitted keys."""
    K, M = counts.shape
    out, pos = {}, 0
    for k in range(K):
        for i in range(M):
            n = int(counts[k, i])
            ks = keys[pos:pos + n]
            assert (vals[pos:pos + n] == i).all()
            assert ((ks >> np.uint64(32)) & np.uint64((1 << bit_k) - 1) == k).all()
            out[(k, i)] = (ks >> np.uint64(32 + bit_k)).astype(np.int64).tolist()
            pos += n
    assert pos == len(keys)
    return out


def region_q(conic, mx, my, xs, ys):
    a, b, c = (float(v) for v in conic)
    dx = xs - float(mx)
    dy = ys - float(my)
    return a * dx * dx + 2 * b * dx * dy + c * dy * dy


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 16)])
def test_bins_are_superset_of_region_and_tight(tile):
    W, H = 100, 70
    TW, TH = tile
    TX, TY = (W + TW - 1) // TW, (H + TH - 1) // TH
    K, M, C = 2, 150, 3
    conic, tau, depth, means = make_inputs(K, M, C, W, H, 11 + TW)
    counts, keys, vals = oracle.mirror_keys(W, H, tile, conic, tau, depth, means)
    bit_k = oracle.ceil_log2(K)
    got = tiles_of(keys, vals, counts, bit_k)
    xs = np.arange(W)[None, :] + 0.5
    ys = np.arange(H)[:, None] + 0.5
    eps = 1e-5
    n_tiles = 0
    for k in range(K):
        for i in range(M):
            tl = got[(k, i)]
            assert tl == sorted(set(tl))  # ascending, no duplicates
            n_tiles += len(tl)
            t_ = float(tau[k, i])
            if not t_ >= 0:
                assert tl == []
                continue
            must, may = set(), set()
            for l in range(C):
                mx, my = means[k, i, l]
                if not np.isfinite(mx):
                    continue
                q = region_q(conic[k, i], mx, my, xs, ys)
                yy, xx = np.nonzero(q <= t_ * (1 - eps) - 1e-6)
                must |= set((yy // TH * TX + xx // TW).tolist())
                # tightness: minimum of q over the tile's continuous band of
                # pixel-centre heights, at each pixel-centre column
                a, b, c = (float(v) for v in conic[k, i])
                for t in range(TX * TY):
                    tx, ty = t % TX, t // TX
                    xc = np.arange(tx * TW, min(W, tx * TW + TW)) + 0.5
                    lo = ty * TH + 0.5 - float(my)
                    hi = min(H, ty * TH + TH) - 0.5 - float(my)
                    dx = xc - float(mx)
                    dy = np.clip(-b * dx / c, lo, hi)
                    qm = a * dx * dx + 2 * b * dx * dy + c * dy * dy
                    if (qm <= t_ * (1 + eps) + 1e-6).any():
                        may.add(t)
            assert must <= set(tl), (k, i)
            assert set(tl) <= may, (k, i)
    assert n_tiles > 200


def test_union_contains_each_view():
    W, H, K, M, C = 120, 80, 3, 100, 4
    conic, tau, depth, means = make_inputs(K, M, C, W, H, 5, spread=3.0)
    _, keys, vals = oracle.mirror_keys(W, H, (16, 16), conic, tau, depth, means)
    counts = oracle.mirror_count(W, H, (16, 16), conic, tau, means)
    union = tiles_of(keys, vals, counts, oracle.ceil_log2(K))
    for l in range(C):
        one = np.ascontiguousarray(means[:, :, l:l + 1, :])
        c1, k1, v1 = oracle.mirror_keys(W, H, (16, 16), conic, tau, depth, one)
        single = tiles_of(k1, v1, c1, oracle.ceil_log2(K))
        for key, tl in single.items():
            assert set(tl) <= set(union[key])


def test_key_layout_eq11():
    W, H, K, M, C = 64, 48, 5, 60, 2
    conic, tau, depth, means = make_inputs(K, M, C, W, H, 9)
    counts, keys, vals = oracle.mirror_keys(W, H, (16, 16), conic, tau, depth, means)
    bit_k = 3  # ceil(log2 5)
    pos = 0
    for k in range(K):
        for i in range(M):
            for _ in range(int(counts[k, i])):
                key = int(keys[pos])
                assert key & 0xFFFFFFFF == int(depth[k, i].view(np.uint32))
                assert (key >> 32) & 0b111 == k
                assert (key >> 35) < 4 * 3
                pos += 1


def test_sorted_list_and_ranges():
    W, H, K, M, C = 90, 60, 3, 200, 3
    conic, tau, depth, means = make_inputs(K, M, C, W, H, 21)
    T = 6 * 4
    r = oracle.mirror_lists(W, H, (16, 16), conic, tau, depth, means)
    ks, lst, ranges = r["keys_sorted"], r["list"], r["ranges"]
    assert len(ks) == int(r["counts"].sum()) > 100
    assert (np.diff(ks.astype(np.float64)) >= 0).all()
    assert (ks[1:] >= ks[:-1]).all()
    same = ks[1:] == ks[:-1]
    assert (lst[1:][same] > lst[:-1][same]).all()  # ties in ascending id
    covered = 0
    bit_k = oracle.ceil_log2(K)
    for t in range(T):
        for k in range(K):
            s, e = ranges[t, k]
            tk = (ks >> np.uint64(32)).astype(np.int64)
            idx = np.nonzero(tk == (t << bit_k | k))[0]
            if len(idx) == 0:
                assert s == e == 0
                continue
            assert s == idx[0] and e == idx[-1] + 1 and e - s == len(idx)
            d = depth[k, lst[s:e]]
            assert (np.diff(d) >= 0).all()  # depth order within a list
            covered += e - s
    assert covered == len(ks)


def test_degenerate_inputs():
    W, H = 32, 32
    conic = np.array([[[1.0, 0.0, 1.0], [1.0, 2.0, 1.0], [1.0, 0.0, 1.0]]], np.float32)
    tau = np.array([[4.0, 4.0, 0.0]], np.float32)
    depth = np.ones((1, 3), np.float32)
    means = np.array([[[[np.nan, 5.0]], [[10.0, 10.0]], [[10.5, 10.5]]]], np.float32)
    counts = oracle.mirror_count(W, H, (16, 16), conic, tau, means)
    # NaN mean -> culled view; det <= 0 -> no region; tau = 0 -> the point
    # itself, which is the centre of pixel (10, 10): one tile
    assert counts.tolist() == [[0, 0, 1]]
