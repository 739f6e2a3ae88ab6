"""Oracle results at the benchmarked sizes, computed once per test session and shared by the
full-vector parity tests of several files (each costs about a minute of host time)."""
import functools

import synth


@functools.lru_cache(maxsize=None)
def cg_p3_64():
    """(xyz, cells, u, y) for the CG P3 Laplacian on the 64^3 Kuhn cube (1,572,864 cells, 7,189,057
    DoFs; interior jitter 0.2h): u ~ U[-1, 1] in the oracle's canonical numbering and y = A u by the
    oracle's cell loop (Eq. 3)."""
    from oracle import cg, topology

    xyz, cells = synth.kuhn_cube(64, jitter=0.2, seed=synth.SEEDS["jitter"])
    dofs, keys = topology.cg_numbering(cells, 3)
    u = synth.uniform_vector(keys.shape[0], synth.SEEDS["u"])
    y = cg.apply(xyz, cells, u, 3, dofs=dofs)
    return xyz, cells, u, y


@functools.lru_cache(maxsize=None)
def dg_p2_48():
    """(xyz, cells, u, y) for the SIPG P2 operator on the 48^3 Kuhn cube (663,552 cells, 6,635,520
    DoFs): u ~ U[-1, 1] per cell in the user's cell order and y = A u by the oracle (Eq. 5)."""
    from oracle import dg

    xyz, cells = synth.kuhn_cube(48, jitter=0.2, seed=synth.SEEDS["jitter"])
    u = synth.uniform_vector(cells.shape[0] * 10, synth.SEEDS["u"])
    y = dg.apply(xyz, cells, u, 2)
    return xyz, cells, u, y
