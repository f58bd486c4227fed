"""Host-side checks of the seeded input generators (no GPU)."""

import math

from sem_inputs import serving


def test_serving_boxes_are_near_cubic():
    # elements of bounded aspect ratio: a 1 x 1 x E box of the unit cube has
    # elements 1/E thick, which no Jacobi-PCG solves in 20,000 iterations
    for seed in (1, 4, 9):
        for r in serving.request_stream(seed=seed, count=200, rate=10.0):
            d = r["desc"]
            if d["kind"] != "box":
                continue
            dims = sorted((d["nx"], d["ny"], d["nz"]))
            assert dims[2] <= 2 * dims[0], d


def test_serving_sizes_track_the_target():
    for E in (512, 777, 1381, 4096, 9000, 32768):
        d = serving._box_near(E)
        assert abs(math.log(d["nx"] * d["ny"] * d["nz"] / E)) < 0.05


def test_serving_pipes_have_near_isotropic_elements():
    # choosing the cross-section by element count alone gave 2 x 1 sections
    # with ~800 axial layers (aspect ~50); one such request did not converge
    for seed in (1, 4, 9):
        for r in serving.request_stream(seed=seed, count=200, rate=10.0):
            d = r["desc"]
            if d["kind"] != "pipe":
                continue
            assert serving.pipe_aspect(d["nc"], d["nr"], d["nzp"]) <= 4.0, d
    for E in (512, 777, 1381, 4096, 9000, 20000, 32768):
        d = serving._pipe_near(E)
        n = d["nc"] * (d["nc"] + 4 * d["nr"]) * d["nzp"]
        assert abs(math.log(n / E)) < math.log(1.1)
