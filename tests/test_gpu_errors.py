"""Error behaviour of the C ABI on the GPU: invalid arguments, and a bounded
device-side wait that expires (no trap, no hang: CTA 0 leaves before the first
grid barrier, the other CTAs' wait runs out after the set bound)."""
import numpy as np
import pytest

import paper_1803_03922_gb300 as bfs
from tests.gpu_util import gpu_bfs, gpu_graph, need_cuda

pytestmark = pytest.mark.gpu


def test_invalid_arguments():
    need_cuda()
    with pytest.raises(bfs.BfsError) as e:
        gpu_graph(4, np.array([0, 5], np.int32), np.array([1, 2], np.int32))
    assert e.value.code == bfs.BFS_ERR_INVALID
    with pytest.raises(bfs.BfsError) as e:
        gpu_graph(0, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert e.value.code == bfs.BFS_ERR_INVALID
    with pytest.raises(bfs.BfsError) as e:
        gpu_graph(4, np.array([0], np.int32), np.array([1], np.int32), th=-1)
    assert e.value.code == bfs.BFS_ERR_INVALID
    g = gpu_graph(4, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    for s in (-1, 4):
        with pytest.raises(bfs.BfsError) as e:
            g.run(s)
        assert e.value.code == bfs.BFS_ERR_INVALID
    with pytest.raises(bfs.BfsError):
        g.set_options(schedule=99)


def test_bounded_wait_expires_and_context_survives():
    torch = need_cuda()
    src = np.arange(0, 999, dtype=np.int32)
    dst = src + 1
    g = gpu_graph(1000, src, dst, th=4)
    g.set_options(test_skip_barrier=1, barrier_timeout_ms=50)
    with pytest.raises(bfs.BfsError) as e:
        g.run(0, stats=True)
    assert e.value.code == bfs.BFS_ERR_TIMEOUT
    # async form: the status is reported by bfs_wait
    d = torch.empty(1000, dtype=torch.int32, device="cuda")
    p = torch.empty(1000, dtype=torch.int32, device="cuda")
    g.run(0, d, p)
    with pytest.raises(bfs.BfsError) as e:
        g.wait()
    assert e.value.code == bfs.BFS_ERR_TIMEOUT
    # the next normal run on the same graph and context is correct
    g.set_options()
    dd, pp = gpu_bfs(g, 0)
    assert (dd == np.arange(1000)).all() and pp[0] == 0 and (pp[1:] == np.arange(999)).all()
    g.wait()
