"""The swarm's random streams at volume: about 10^7 Philox draws (4 calls of
4096 particles x 640 dimensions, with node ids, iterations, keys and
purposes spanning their ranges) bit-identical between the GPU and the
oracle, and uniform (chi-square over 256 cells)."""
import numpy as np
import pytest

import oracle as O
from tests.gpu_util import context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = context()
    yield c
    c.close()


@pytest.mark.parametrize("seed,uid,t,purpose", [
    (1, 0, 0, 1), (0x0123456789ABCDEF, 2**32 - 1, 2**32 - 1, 4),
    (2**63 + 12345, 65536 * 200 + 17, 100, 3), (99, 7, 2**31 + 5, 255)])
def test_ten_million_draws_bitwise(ctx, seed, uid, t, purpose):
    from scipy import stats
    P, d = 4096, 640
    g = ctx.swarm_uniforms(seed, uid, t, P, d, purpose)
    o = O.swarm_uniforms(seed, uid, t, P, d, purpose)
    assert np.array_equal(g.view(np.uint32), o.view(np.uint32))
    counts = np.bincount((g.ravel() * 256).astype(np.int64), minlength=256)
    assert stats.chisquare(counts).pvalue > 1e-4
