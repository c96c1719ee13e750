"""The standalone device Hines solve (mm_hines_solve, Algorithm 1 on a batch
of trees) against the oracle's Algorithm 1 and dense Gaussian elimination."""
import numpy as np
import pytest

import oracle
from paper_2005_06332_gb300 import mm, netgen

pytestmark = pytest.mark.gpu


def _batch(seed, n_trees, max_n, p_branch=0.3):
    rng = np.random.default_rng(seed)
    sizes = rng.integers(1, max_n + 1, n_trees)
    off = np.zeros(n_trees + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    par, a, b, c, r = [], [], [], [], []
    for n in sizes:
        p = netgen.random_tree(rng, int(n), p_branch)
        aa = -rng.uniform(0.1, 1.0, n)
        cc = -rng.uniform(0.1, 1.0, n)
        aa[0] = cc[0] = 0.0
        bb = rng.uniform(0.5, 2.0, n) + 2.0 * (np.abs(aa) + np.abs(cc))
        par.append(p); a.append(aa); b.append(bb); c.append(cc); r.append(rng.normal(size=n))
    return off, np.concatenate(par), *(np.concatenate(v) for v in (a, b, c, r))


def _gpu(off, par, a, b, c, r):
    import torch
    dev = torch.device("cuda", 0)
    t = lambda v, dt: torch.as_tensor(v, dtype=dt, device=dev)
    x = mm.hines_solve(t(off, torch.int64), t(par, torch.int32), t(a, torch.float64), t(b, torch.float64),
                       t(c, torch.float64), t(r, torch.float64))
    return x.cpu().numpy()


@pytest.mark.parametrize("seed,n_trees,max_n", [(0, 1, 1), (1, 7, 16), (2, 300, 16), (3, 40, 700)])
def test_batch_solve_matches_oracle_algorithm_1(seed, n_trees, max_n):
    off, par, a, b, c, r = _batch(seed, n_trees, max_n)
    x = _gpu(off, par, a, b, c, r)
    for k in range(n_trees):
        s, e = off[k], off[k + 1]
        ref = oracle.hines_solve(a[s:e], b[s:e], c[s:e], r[s:e], par[s:e])
        np.testing.assert_allclose(x[s:e], ref, rtol=1e-12, atol=1e-14)


def test_batch_solve_rejects_bad_parent():
    import torch
    off, par, a, b, c, r = _batch(4, 3, 10)
    par = par.copy()
    par[off[1] + 1] = 5  # parent after child
    with pytest.raises(mm.MMError) as e:
        _gpu(off, par, a, b, c, r)
    assert e.value.status == mm.MM_EINVAL


def _raw_call(fn, off, par, a, b, c, r, n_comp):
    """Call an entry point through the C-ABI with an explicit n_comp (the
    device buffers hold every entry of the offsets, whatever n_comp says)."""
    import ctypes as C
    import torch
    dev = torch.device("cuda", 0)
    t = [torch.as_tensor(v, dtype=dt, device=dev)
         for v, dt in zip((off, par, a, b, c, r), (torch.int64, torch.int32) + (torch.float64,) * 4)]
    x = torch.full_like(t[5], float("nan"))
    st = fn(len(off) - 1, int(n_comp), t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), t[3].data_ptr(),
            t[4].data_ptr(), t[5].data_ptr(), x.data_ptr(), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, x.cpu().numpy()


def test_batch_solve_rejects_offsets_outside_n_comp():
    """A tree whose entry range reaches past n_comp (or runs backwards) is
    rejected with MM_EINVAL before any of its entries is touched; the other
    trees are still solved."""
    L = mm.load()
    off, par, a, b, c, r = _batch(5, 6, 12)
    st, x = _raw_call(L.mm_hines_solve, off, par, a, b, c, r, off[-1] - 1)
    assert st == mm.MM_EINVAL
    for k in range(5):
        s, e = off[k], off[k + 1]
        np.testing.assert_allclose(x[s:e], oracle.hines_solve(a[s:e], b[s:e], c[s:e], r[s:e], par[s:e]),
                                   rtol=1e-12, atol=1e-14)
    assert np.all(np.isnan(x[off[5]:]))  # the rejected tree was not written
    bad = off.copy()
    bad[2], bad[3] = off[3], off[2]  # tree 1 takes in tree 2's root; tree 2 runs backwards
    st, _ = _raw_call(L.mm_hines_solve, bad, par, a, b, c, r, off[-1])
    assert st == mm.MM_EINVAL
