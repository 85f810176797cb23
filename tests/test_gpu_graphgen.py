"""The device generator reproduces the host twin bit for bit (scales 10-16)."""
import numpy as np
import pytest

import graphgen
from tests.gpu_util import need_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scale", [10, 13, 16])
def test_rmat_device_equals_host(scale):
    need_cuda()
    hs, hd = graphgen.rmat_host(scale, seed=scale * 7 + 1)
    ds, dd = graphgen.rmat_device(scale, seed=scale * 7 + 1)
    assert np.array_equal(ds.cpu().numpy(), hs) and np.array_equal(dd.cpu().numpy(), hd)
    hm = graphgen.nonisolated_mask_host(1 << scale, hs, hd)
    dm = graphgen.nonisolated_mask_device(1 << scale, ds, dd)
    assert np.array_equal(dm.cpu().numpy(), hm)


def test_er_device_equals_host():
    need_cuda()
    hs, hd = graphgen.er_host(3000, 50000, seed=9)
    ds, dd = graphgen.er_device(3000, 50000, seed=9)
    assert np.array_equal(ds.cpu().numpy(), hs) and np.array_equal(dd.cpu().numpy(), hd)
