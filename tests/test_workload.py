"""The seeded input generators: the tensor-grid evaluation of the bump field equals
the pointwise definition, and sequences are reproducible and seed-dependent."""
import numpy as np

from workload import BumpSequence, load_sequence, lumped_nodal_volumes, make_mesh


def test_bump_field_on_grid_equals_pointwise():
    m = make_mesh(12, 4, 1.3, 20.0)
    x0, x1, y0, y1, z0, z1 = m.free_box
    for seed in (1, 9):
        seq = BumpSequence(seed)
        for t in (0, 7):
            a = seq.f(m.free_node_coords(), t)
            b = seq.f_grid(m.xc[x0:x1], m.yc[y0:y1], m.zc[z0:z1], t)
            assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()


def test_sequence_reproducible_and_seeded():
    m = make_mesh(8, 4, 1.0, None)
    a = load_sequence(m, 3, 4)
    assert np.array_equal(a, load_sequence(m, 3, 4))
    assert np.array_equal(a[2:], load_sequence(m, 3, 2, start=2))
    assert not np.allclose(a, load_sequence(m, 4, 4))
    # lumped volumes of all nodes (free and Dirichlet) sum to the unit cube
    assert lumped_nodal_volumes(m).sum() <= 1.0 + 1e-12
