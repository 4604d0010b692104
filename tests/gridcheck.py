"""Helpers of the GPU tests: an oracle grid for a synthetic workload and a
voxel-by-voxel comparison that reports the first mismatch.

The CUDA side never feeds the oracle: both are driven with the same seeded
frames from synth/, and every grid the library produces is compared with
the oracle's after the same calls.
"""
import numpy as np

from oracle import OracleGrid, OracleParams


def oracle_grid(w, literal=0):
    """An oracle grid with workload w's parameters, centred on its first
    frame's robot position (as the library grid made for w)."""
    g = w.grid
    return OracleGrid(OracleParams(tuple(g.n), g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf,
                                   literal), w.frames[0].robot_pos)


def assert_same(got, ref, what):
    """got and ref: (Nz, Ny, Nx) voxel codes.  Bit-exact or an error naming
    the first differing voxel and the counts of (gpu, oracle) state pairs."""
    got = np.asarray(got).reshape(ref.shape)
    bad = np.argwhere(got != ref)
    if len(bad):
        z, y, x = bad[0]
        pairs = {}
        for b in bad[:100000]:
            k = (int(got[tuple(b)]), int(ref[tuple(b)]))
            pairs[k] = pairs.get(k, 0) + 1
        raise AssertionError("%s: %d voxels differ; first (x=%d, y=%d, z=%d) gpu=%d oracle=%d; "
                             "(gpu, oracle) pair counts %s" % (what, len(bad), x, y, z, got[z, y, x],
                                                               ref[z, y, x], pairs))


def assert_grid(got, origin, og, what):
    """A library grid (flat codes and origin) against an OracleGrid."""
    assert list(origin) == list(og.o), (what, list(origin), list(og.o))
    assert_same(got, og.loc, what)
