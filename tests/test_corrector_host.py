"""Host-side parts of the corrector workflow (no GPU): the training shapes keep away from the
held-out radii and stay inside the stated ranges, the seeded draw is repeatable, the masks
have the grid's shape, and the spectrum error is the stated relative L1 distance."""
import numpy as np

from paper_2304_03306_gb300 import corrector as C


def test_training_shapes_avoid_held_out_radii_and_respect_ranges():
    shapes = C.training_shapes(400, seed=3)
    assert len(shapes) == 400
    assert shapes == C.training_shapes(400, seed=3)
    circles = [s for s in shapes if s[0] == "circle"]
    dumbbells = [s for s in shapes if s[0] == "dumbbell"]
    assert circles and dumbbells
    for _, R in circles:
        assert 5.0 <= R <= 7.0 and min(abs(R - h) for h in C.HELD_OUT) >= 0.1
    for _, R, D in dumbbells:
        assert 2.8 <= R <= 3.5 and 1.0 <= D / R <= 1.9


def test_masks_and_spectrum_error():
    m = C.mask_for(("circle", 5.5), C.COARSE)
    assert m.shape == (C.COARSE["n"],) * 2 and m.dtype == np.uint8
    d = C.mask_for(("dumbbell", 3.0, 4.5), C.FINE)
    assert d.shape == (C.FINE["n"],) * 2
    ref = np.array([1.0, 2.0, 3.0])
    assert C.spectrum_error(ref, ref) == 0.0
    assert abs(C.spectrum_error(ref * 1.1, ref) - 0.1) < 1e-12
    assert C.NBINS == C.COARSE["n"] // 4 + 1
