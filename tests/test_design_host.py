"""Host-side bookkeeping of the design update (no GPU): the design's bounding box and the
placement of design values in it."""
import numpy as np

from paper_2412_16845_gb300.adjoint import design_box


def test_design_box_places_values_on_their_cells():
    rng = np.random.default_rng(3)
    nx, ny = 37, 23
    design = np.sort(rng.choice(nx * ny, size=40, replace=False))
    box, index, cells = design_box(design, nx)
    x0, x1, y0, y1 = box
    xs, ys = design % nx, design // nx
    assert (x0, x1, y0, y1) == (xs.min(), xs.max() + 1, ys.min(), ys.max() + 1)
    assert cells.size == (x1 - x0) * (y1 - y0)
    eps = rng.uniform(1, 2, nx * ny)
    vals = rng.uniform(3, 4, design.size)
    boxvals = eps[cells].copy()
    boxvals[index] = vals
    full = eps.copy()
    full[design] = vals
    # the box, written back row by row, is the full eps with the design replaced
    out = eps.copy()
    out.reshape(ny, nx)[y0:y1, x0:x1] = boxvals.reshape(y1 - y0, x1 - x0)
    assert np.array_equal(out, full)


def test_design_box_of_a_rectangle_is_the_rectangle():
    nx = 16
    ii, jj = np.arange(4, 9), np.arange(2, 7)
    design = (jj[:, None] * nx + ii[None, :]).ravel()
    box, index, cells = design_box(design, nx)
    assert box == (4, 9, 2, 7)
    assert np.array_equal(index, np.arange(design.size))
    assert np.array_equal(cells, design)
