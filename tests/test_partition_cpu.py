"""Host logic of the iterative solver: the lattice grouping behind its coarse model and block-Jacobi
blocks (gdm_lattice_partition, host memory only, no GPU). Checked against definitions written out here:
the permutation sorts the cells by the 3D Morton (bit-interleaved) key of their lattice indices, every
coarse cell is one 2 x 2 x 2 lattice cube and holds a contiguous run of the permuted cells, and the
coarse cells follow the fine order."""
import numpy as np
import pytest

import gdm_workloads as W


@pytest.fixture(scope="module")
def B():
    from paper_2505_09545_gb300 import binding
    binding.lib()
    return binding


def morton(ijk):
    """Interleave the bits of (i, j, k): bit b of i goes to 3b, of j to 3b + 1, of k to 3b + 2."""
    key = 0
    for b in range(21):
        for a in range(3):
            key |= ((int(ijk[a]) >> b) & 1) << (3 * b + a)
    return key


def lattice(pos, step):
    return np.floor((pos - pos.min(axis=0)) / step + 0.5).astype(np.int64)


@pytest.mark.parametrize("case", ["cuboid", "blob", "sphere", "jitter"])
def test_partition_invariants(B, case):
    rng = np.random.default_rng(5)
    if case == "cuboid":
        pos, step = W.cuboid_cells(9, 7, 5, 10.0), 10.0
    elif case == "blob":
        pos, step = W.eden_blob(700, 15.0, rng), 15.0
    elif case == "sphere":
        pos, step = W.sphere_cells(60.0, 10.0), 10.0
    else:  # positions off the lattice by up to a quarter step still group by rounding
        pos, step = W.cuboid_cells(6, 6, 6, 10.0) + rng.uniform(-2.4, 2.4, (216, 3)), 10.0
    n = len(pos)
    perm, parent, coff = B.lattice_partition(pos, step, block_cells=64)
    # a permutation sorted by the Morton key of the lattice indices
    assert sorted(perm.tolist()) == list(range(n))
    ijk = lattice(pos, step)
    keys = [morton(ijk[p]) for p in perm]
    assert keys == sorted(keys)
    # coarse cells: contiguous runs, one 2x2x2 cube each, offsets consistent with the parents
    nc = len(coff) - 1
    assert coff[0] == 0 and coff[-1] == n and np.all(np.diff(coff) >= 1) and np.all(np.diff(coff) <= 8)
    for c in range(nc):
        run = perm[coff[c]:coff[c + 1]]
        assert np.all(parent[coff[c]:coff[c + 1]] == c)
        cubes = {tuple(v) for v in ijk[run] // 2}
        assert len(cubes) == 1
    # every cube appears once
    assert len({tuple(v) for v in ijk // 2}) == nc


def test_partition_of_a_full_aligned_cube(B):
    """An 8 x 8 x 8 lattice cube: 64 coarse cells of exactly 8 children, and Morton order makes each
    run of 64 cells a 4 x 4 x 4 sub-cube (the blocks of 64 cells are compact)."""
    pos = W.cuboid_cells(8, 8, 8, 10.0)
    perm, parent, coff = B.lattice_partition(pos, 10.0, block_cells=64)
    assert len(coff) - 1 == 64 and np.all(np.diff(coff) == 8)
    ijk = lattice(pos, 10.0)
    for b in range(8):
        sub = ijk[perm[64 * b:64 * (b + 1)]]
        assert np.all(sub.max(axis=0) - sub.min(axis=0) == 3)


def test_partition_rejects_bad_input(B):
    pos = W.cuboid_cells(2, 2, 2, 10.0)
    with pytest.raises(B.GDMError):
        B.lattice_partition(pos, 0.0)
    bad = pos.copy()
    bad[3, 1] = np.nan
    with pytest.raises(B.GDMError):
        B.lattice_partition(bad, 10.0)
    one, par, coff = B.lattice_partition(np.zeros((1, 3)), 10.0)
    assert one.tolist() == [0] and par.tolist() == [0] and coff.tolist() == [0, 1]
