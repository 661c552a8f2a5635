"""GPU test of nbr_build_noalloc, the neighbour build for callers that cannot
allocate device memory (a host framework that owns every device allocation,
a plug-in limited to the buffers it is given). Its scratch is a fixed static device array; these checks call it
through the C ABI and compare its lists with nbr_build's, bit for bit, on
consecutive calls that reuse that array."""
import ctypes as ct

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2602_14975_gb300 import _lib as L
from paper_2602_14975_gb300 import core
from paper_2602_14975_gb300 import synth as S

pytestmark = pytest.mark.gpu

MAX_ATOMS = 131072


def _noalloc(dsys, r_list, capacity):
    row = torch.full((dsys.n_atoms + 1,), -7, dtype=torch.int32, device=dsys.x.device)
    col = torch.full((max(1, capacity),), -7, dtype=torch.int32, device=dsys.x.device)
    s = dsys.struct()
    nb = L.Nbr(ct.c_void_p(row.data_ptr()), ct.c_void_p(col.data_ptr()), capacity, float(r_list))
    n = ct.c_longlong(0)
    st = L.lib().nbr_build_noalloc(ct.byref(s), ct.byref(nb), ct.byref(n),
                                   ct.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, row, col, int(n.value)


def _compare(ctx, dsys, r_list):
    ref = core.nbr_build(ctx, dsys, r_list)
    st, row, col, n = _noalloc(dsys, r_list, ref.n_pairs + 64)
    assert st == L.OK, L.lib().dmts_last_error(None)
    assert n == ref.n_pairs
    assert torch.equal(row, ref.row_ptr)
    assert torch.equal(col[:n], ref.col[:n])


def test_noalloc_matches_nbr_build_on_consecutive_calls():
    cs = S.cons_spec(1, 32, 1)
    ctx = core.Context(cons=(cs, S.cons_weights(cs, 1)))
    water = core.DeviceSystem(S.water_192())
    drops = core.DeviceSystem([S.capped_molecule_in_droplet(n, seed=60 + n) for n in (20, 57, 33)])
    _compare(ctx, water, 5.5)      # first call: sets up the scratch address
    _compare(ctx, drops, 5.5)      # second call reuses the array left by the first
    _compare(ctx, water, 4.5)      # and a third, back to the periodic box
    torch.cuda.synchronize()


def test_noalloc_overflow_then_recovers_and_rejects_oversize():
    water = core.DeviceSystem(S.water_192())
    st, _, _, need = _noalloc(water, 5.5, 100)
    assert st == L.E_NBR_OVERFLOW
    assert need > 100
    st, row, col, n = _noalloc(water, 5.5, need)     # the error word was cleared
    assert st == L.OK and n == need
    big = water.struct()
    big.n_atoms = MAX_ATOMS + 1                        # rejected before any device work
    nb = L.Nbr(ct.c_void_p(row.data_ptr()), ct.c_void_p(col.data_ptr()), n, 5.5)
    nn = ct.c_longlong(0)
    assert L.lib().nbr_build_noalloc(ct.byref(big), ct.byref(nb), ct.byref(nn), None) == L.E_INVALID
    assert b"DMTS_STATIC_MAX_ATOMS" in L.lib().dmts_last_error(None)


def test_noalloc_empty_system_writes_its_row_offset():
    """A system without atoms launches nothing; the call still sets the one
    row offset it owns to 0 (the buffer held -7)."""
    none = S.System("none", np.zeros((0, 3)), np.zeros(0, np.uint8), np.zeros(0, np.int32),
                    np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(3))
    d0 = core.DeviceSystem(none)
    st, row, _, n = _noalloc(d0, 5.5, 16)
    assert st == L.OK, L.lib().dmts_last_error(None)
    assert n == 0 and row.cpu().tolist() == [0]
