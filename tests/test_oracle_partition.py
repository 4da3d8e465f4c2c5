"""Pins of the t-split domain decomposition (oracle.partition): the sub-domain Dslash with
ghost faces, exchanged in process, equals the whole-lattice operator (exactly up to
rounding), for 1, 2 and 4 sub-domains and both parities."""
import numpy as np
import pytest

import synth
from oracle import dslash, partition as part


def _exchange(U_parts, chi_parts, dims_loc):
    P = len(chi_parts)
    fs = [part.faces(c, dims_loc) for c in chi_parts]
    ghost_Ut = [part.last_slice_links(U_parts[(k - 1) % P], dims_loc) for k in range(P)]
    ghost_bwd = [fs[(k - 1) % P][1] for k in range(P)]
    ghost_fwd = [fs[(k + 1) % P][0] for k in range(P)]
    return ghost_Ut, ghost_bwd, ghost_fwd


@pytest.mark.parametrize("dims,P", [((4, 2, 2, 4), 1), ((4, 4, 2, 8), 2), ((2, 4, 4, 8), 4), ((4, 2, 4, 4), 2)])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_partitioned_dslash_equals_whole_lattice(dims, P, out_parity):
    U = synth.gauge_field(dims, "haar", seed=601)
    chi = synth.fermion_field(dims, 1, 602)[0]
    ref = dslash.dslash_eo(U, chi, dims, out_parity)
    dl = part.local_dims(dims, P)
    Up = part.split_gauge(U, dims, P)
    cp = part.split_vec(chi, dims, P)
    gU, gb, gf = _exchange(Up, cp, dl)
    got = part.join_vec([part.dslash_eo_halo(Up[k], gU[k], cp[k], gb[k], gf[k], dl, out_parity)
                         for k in range(P)])
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_split_join_round_trip_and_faces():
    dims = (4, 4, 2, 8)
    v = synth.fermion_field(dims, 2, 603)
    parts = part.split_vec(v, dims, 4)
    assert np.array_equal(part.join_vec(parts), v)
    lo, hi = part.faces(parts[1], part.local_dims(dims, 4))
    Vsh = 4 * 4 * 2 // 2
    assert np.array_equal(lo, v[:, 2 * Vsh:3 * Vsh]) and np.array_equal(hi, v[:, 3 * Vsh:4 * Vsh])
    with pytest.raises(ValueError):
        part.local_dims((4, 4, 4, 6), 2)   # 3 slices per part: odd
