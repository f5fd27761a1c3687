"""The seeded input generators (no method arithmetic): the PyTorch copy of the
counter-based generator draws the same bits as the NumPy one, and the batch
shapes follow their stated recipe."""
import numpy as np
import pytest

import synthetic


@pytest.mark.parametrize("seed,offset,n", [(1, 0, 1000), (7, 12345, 4097), (100, (1 << 35) + 3, 257)])
def test_torch_generator_matches_numpy(seed, offset, n):
    torch = pytest.importorskip("torch")
    a = synthetic.uniform01(seed, n, offset=offset)
    b = synthetic.uniform01_torch(seed, n, offset=offset).numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_torch_planes_match_uniform_field():
    pytest.importorskip("torch")
    shape = (20, 12, 16)
    f = synthetic.uniform_field(shape, 9)
    for z0, z1 in ((0, 20), (0, 8), (8, 12), (12, 20)):
        g = synthetic.uniform_field_planes_torch(shape, 9, z0, z1).numpy()
        assert np.array_equal(g.view(np.uint32), f[z0:z1].view(np.uint32)), (z0, z1)


def test_batch_shapes_recipe():
    sh = synthetic.batch_shapes(64)
    assert len(sh) == 64
    assert [s for s, _ in sh[:4]] == ["heat", "wave", "heat", "wave"]
    sides = np.array([d for _, dims in sh for d in dims])
    assert sides.min() >= 64 and sides.max() <= 384 and np.all(sides % 16 == 0)
    assert len(set(sides.tolist())) > 10  # uneven
    assert sh == synthetic.batch_shapes(64)  # seeded


def test_uniform_field_box_is_a_window_of_the_field():
    shape = (20, 24, 28)
    full = synthetic.uniform_field(shape, 7)
    for (z0, y0, x0, n) in ((0, 0, 0, 8), (5, 9, 13, 7), (12, 16, 20, 8)):
        box = synthetic.uniform_field_box(shape, 7, z0, y0, x0, n)
        assert np.array_equal(box, full[z0:z0 + n, y0:y0 + n, x0:x0 + n])
