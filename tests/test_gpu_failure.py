"""Failure detection on the GPU without a fault: a kernel waits on an mbarrier
that nothing completes; the library's bounded wait gives up after about a
second, reports through the device status word, and the host sees
NDF_ERR_TIMEOUT.  The context stays usable and the next calls succeed."""
import time

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(ndf_mod, ctx, tiny_field, tiny_ref):
    t0 = time.perf_counter()
    st = ndf_mod.ndf_selftest_timeout(ctx)
    elapsed = time.perf_counter() - t0
    assert st == ndf_mod.NDF_ERR_TIMEOUT
    assert 0.5 <= elapsed <= 30.0, elapsed
    assert "bounded device wait" in ndf_mod.ndf_last_error(ctx)
    # the status word was cleared and the context works
    M, Z, Y, X = tiny_field.shape
    fid = ndf_mod.ndf_load_ensemble(ctx, tiny_field, M, Z, Y, X)
    out = np.empty(tiny_field[0].size, np.float32)
    ndf_mod.ndf_pearson(ctx, fid, fid, tiny_ref, out)
    assert np.abs(out - oracle.pearson_volume(tiny_field, tiny_field, tiny_ref)).max() <= 1e-5
    ndf_mod.ndf_mi_ksg(ctx, fid, fid, tiny_ref, 4, out)
    ndf_mod.ndf_synchronize(ctx)
    ndf_mod.ndf_free_ensemble(ctx, fid)
