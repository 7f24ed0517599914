"""Pins of the oracle's panel functions: view index (Sec. 3.1, Eq. 1-3),
view-coherent remap (Sec. 4.3, Eq. 8) and clustering (Appendix B.1)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2605_04509_gb300 import synth


def _exact_view(x, y, u, n, tan_slant: Fraction, pitch: Fraction, k_off: Fraction):
    d = 3 * x + u + 3 * y * tan_slant - k_off
    xoff = d - pitch * (d // pitch)
    r = n * xoff / pitch
    return min(max(r.numerator // r.denominator, 0), n - 1)


def test_view_index_exact_rationals_tiny_panel():
    # Eq. 1-3 evaluated in exact rational arithmetic on the 256x144 panel with
    # tan(alpha) = 1/6 and L_x = 9/2; one subpixel in nine sits exactly on a
    # view boundary, so the FP64 operation order is checked there too.
    p = synth.WORKLOADS["tiny"].panel
    V = oracle.view_index(p)
    assert V.shape == (p.height, p.width, 3)
    ta, L = Fraction(1, 6), Fraction(9, 2)
    on_boundary = 0
    for y in range(p.height):
        for x in range(p.width):
            for u in range(3):
                d = 3 * x + u + 3 * y * ta
                r = 8 * (d - L * (d // L)) / L
                on_boundary += r.denominator == 1
                assert V[y, x, u] == _exact_view(x, y, u, 8, ta, L, Fraction(0))
    assert on_boundary == 12288


def test_view_index_exact_rationals_offset_panel():
    # dyadic parameters, non-zero K_offset (negative d on the left edge)
    W, H, N = 37, 23, 13
    ta, L, koff = Fraction(1, 4), Fraction(21, 4), Fraction(3, 2)
    V = oracle.view_index(synth.Panel(W, H, N, float(ta), float(L), float(koff)))
    for y in range(H):
        for x in range(W):
            for u in range(3):
                assert V[y, x, u] == _exact_view(x, y, u, N, ta, L, koff)


def test_view_index_no_slant_pitch_equals_views():
    # Special case: no slant and a pitch of exactly N subpixels makes the view
    # cycle through 0..N-1 along each row, one per subpixel: j = (3x+u) mod N.
    W, H, N = 40, 5, 7
    V = oracle.view_index(synth.Panel(W, H, N, 0.0, float(N), 0.0))
    x = np.arange(W)[None, :, None]
    u = np.arange(3)[None, None, :]
    expect = np.broadcast_to((3 * x + u) % N, (H, W, 3))
    assert np.array_equal(V, expect)


def test_view_index_slant_shifts_rows():
    # With tan(alpha) = 1/3 each row is the previous one shifted by one
    # subpixel: V[y+1] at subpixel s equals V[y] at subpixel s+1.
    W, H, N = 30, 6, 9
    V = oracle.view_index(synth.Panel(W, H, N, 1.0 / 3.0, 4.5, 0.0))
    flat = V.reshape(H, W * 3).astype(int)
    # d = 3x+u + y (exactly), so rows shift by one subpixel per row
    assert np.array_equal(flat[1:, :-1], flat[:-1, 1:])


def test_view_index_periodic_and_balanced():
    # d advances by L_x every L_x subpixels, so with L_x = 9/2 the pattern
    # repeats every 9 subpixels (3 pixels); views are used near-uniformly.
    V = oracle.view_index(synth.Panel(90, 4, 8, 0.0, 4.5, 0.0)).reshape(4, -1)
    assert np.array_equal(V[:, 9:], V[:, :-9])
    counts = np.bincount(V.reshape(-1), minlength=8)
    assert counts.min() > 0 and counts.max() - counts.min() <= V.size // 9 + 1


def test_view_index_rejects_bad_panels():
    with pytest.raises(RuntimeError):
        oracle.view_index(synth.Panel(8, 8, 256, 0.0, 4.0))
    with pytest.raises(RuntimeError):
        oracle.view_index(synth.Panel(8, 8, 8, 0.0, 0.0))


@pytest.mark.parametrize("W,H,TW,TH,C", [(256, 144, 16, 16, 8), (50, 37, 16, 16, 3),
                                         (33, 20, 8, 8, 1), (70, 19, 32, 16, 4)])
def test_remap_is_stable_view_sort(W, H, TW, TH, C):
    N = 11
    V = oracle.view_index(synth.Panel(W, H, N, 0.2027, 5.3, 0.7))
    psi, n_sub, seg = oracle.remap(V, N, TW, TH, C)
    TX = (W + TW - 1) // TW
    K = oracle.num_clusters(N, C)
    for t in range(psi.shape[0]):
        tx, ty = t % TX, t // TX
        w = min(TW, W - tx * TW)
        h = min(TH, H - ty * TH)
        assert n_sub[t] == 3 * w * h  # ragged edge tiles hold in-panel subpixels only
        loc = psi[t, : n_sub[t]].astype(int)
        yl, rem = loc // (3 * TW), loc % (3 * TW)
        xl, u = rem // 3, rem % 3
        assert (xl < w).all() and (yl < h).all()
        # a permutation of the tile's subpixels
        assert len(set(loc.tolist())) == n_sub[t]
        views = V[ty * TH + yl, tx * TW + xl, u].astype(int)
        # Eq. 8: V[Psi(r)] <= V[Psi(r+1)]
        assert (np.diff(views) >= 0).all()
        # stable: row-major order kept among equal views
        same = np.diff(views) == 0
        assert (np.diff(loc)[same] > 0).all()
        # seg marks where each cluster's run starts
        for k in range(K + 1):
            assert seg[t, k] == np.searchsorted(views // C, k, side="left")


def test_clusters_appendix_b1_tables():
    # Appendix B.1: contiguous clusters of |V_k| views, the last one padded
    # with v_{N-1}, representative at local index floor(|V_k|/2).
    slot, rep = oracle.clusters(45, 8)
    assert slot.shape == (6, 8)
    assert slot[0].tolist() == [0, 1, 2, 3, 4, 5, 6, 7]
    assert slot[5].tolist() == [40, 41, 42, 43, 44, 44, 44, 44]
    assert rep.tolist() == [4, 12, 20, 28, 36, 44]
    slot, rep = oracle.clusters(100, 8)
    assert slot.shape[0] == 13 and rep[-1] == 99 and rep[-2] == 92
    slot, rep = oracle.clusters(71, 18)
    assert rep.tolist() == [9, 27, 45, 63]
    slot, rep = oracle.clusters(8, 8)
    assert rep.tolist() == [4]
    slot, rep = oracle.clusters(5, 1)
    assert rep.tolist() == [0, 1, 2, 3, 4]
    slot, rep = oracle.clusters(3, 8)  # one cluster larger than the view count
    assert slot[0].tolist() == [0, 1, 2, 2, 2, 2, 2, 2] and rep.tolist() == [2]
