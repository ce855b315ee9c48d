"""The 14-cycle circuit's recorded path and slicing are what the seeded generators give
(tn_inputs/search_paths.py records them): the greedy run of the recorded parameters has
the recorded cost, and the greedy slicer picks the recorded labels, the first seven of
which bring every slice's largest intermediate to 2^30 elements."""
import pytest

from tn_inputs import greedy, workloads


def test_rc40c14_path_cost():
    w = workloads.rc40c14()
    assert len(w.net.modes) == 316 and len(w.path.pairs) == 315
    assert greedy.path_log2_flops(w.net, w.path) == pytest.approx(50.8119, abs=1e-3)
    assert greedy.path_peak(w.net, w.path) == 37.0  # unsliced: 2^37 elements


def test_rc40c14_slicing_reproduces():
    w = workloads.rc40c14()
    sub = greedy.greedy_slicer(w.net, w.path, -1.0, max_slices=9)
    assert tuple(sub) == workloads.RC40C14_SUBSLICED
    assert greedy.path_peak(w.net, w.path, sub[:6]) > 30.0
    assert greedy.path_peak(w.net, w.path, sub[:7]) == 30.0
    assert greedy.path_peak(w.net, w.path, sub) == 29.0
    assert workloads.rc40c14().n_slices == 128 and workloads.rc40c14sub().n_slices == 512


def test_rc40c14_pieces_cover_each_slice():
    """Slice s of the 7-label slicing is the union of pieces 4s..4s+3 of the 9-label one:
    the first seven sliced labels take the same values (mixed radix, first label most
    significant)."""
    import oracle.core as core
    w, sub = workloads.rc40c14(), workloads.rc40c14sub()
    for s in (0, 37, 127):
        a = core.slice_assignment(w.net, w.sliced, s)
        for j in range(4):
            b = core.slice_assignment(sub.net, sub.sliced, 4 * s + j)
            assert all(b[x] == a[x] for x in w.sliced)
