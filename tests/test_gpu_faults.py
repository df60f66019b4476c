"""Failure detection without a GPU fault (needs a GPU).

* A bounded device wait that runs out ends in a status: the self-test kernel
  waits on an mbarrier nothing arrives on, gives up after its clock budget and
  the call returns EDPC_ETIMEOUT; the context then still compresses and
  decompresses.
* A device allocation that cannot be satisfied (the FDMs of 65535 streams of
  the "w/o LTE" model with F = 1024: about 0.8 TB) returns EDPC_ENOMEM and
  leaves the device usable.
"""
import numpy as np
import pytest

pytest.importorskip("torch")

import paper_2507_18969_gb300 as edpc  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _round_trip_still_works():
    x = synth.markov_bytes(5000, 1, 0.05, 2)
    c = edpc.make_cfg(streams=4, context=8, embed_dim=8, latent=64, hidden=64, precision=edpc.EDPC_BF16)
    assert np.array_equal(edpc.decompress(edpc.compress(x, c)), x)


def test_bounded_wait_expires_with_a_status():
    for _ in range(2):
        with pytest.raises(edpc.EdpcError) as e:
            edpc.selftest_wait_timeout()
        assert e.value.code == 6  # EDPC_ETIMEOUT
    _round_trip_still_works()


def test_device_allocation_failure_is_enomem():
    c = edpc.make_cfg(streams=65535, context=64, embed_dim=16, latent=0, hidden=64, blocks=2)
    with pytest.raises(edpc.EdpcError) as e:
        edpc.Model(c, 65535)
    assert e.value.code == 2  # EDPC_ENOMEM
    _round_trip_still_works()
