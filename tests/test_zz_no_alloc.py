"""mm_hines_solve_noalloc: the batched Algorithm 1 solve for callers that may
not allocate device memory (its scratch is a fixed device array inside the
library).  Called through the C-ABI twice in a row and checked against the
allocating mm_hines_solve on the same inputs.  This file runs last so that a
failure here never hides another test's result."""
import ctypes as C

import numpy as np
import pytest

from paper_2005_06332_gb300 import mm, netgen

pytestmark = pytest.mark.gpu

MAX_COMPS = 1 << 20


def _inputs(seed, n_trees, max_n):
    rng = np.random.default_rng(seed)
    sizes = rng.integers(1, max_n + 1, n_trees)
    off = np.zeros(n_trees + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    par, a, b, c, r = [], [], [], [], []
    for n in sizes:
        p = netgen.random_tree(rng, int(n), 0.3)
        aa = -rng.uniform(0.1, 1.0, n)
        cc = -rng.uniform(0.1, 1.0, n)
        aa[0] = cc[0] = 0.0
        bb = rng.uniform(0.5, 2.0, n) + 2.0 * (np.abs(aa) + np.abs(cc))
        par.append(p); a.append(aa); b.append(bb); c.append(cc); r.append(rng.normal(size=n))
    return off, np.concatenate(par), *(np.concatenate(v) for v in (a, b, c, r))


def _device(arrays):
    import torch
    dev = torch.device("cuda", 0)
    dts = (torch.int64, torch.int32) + (torch.float64,) * 4
    return [torch.as_tensor(v, dtype=dt, device=dev) for v, dt in zip(arrays, dts)]


def _call(fn, t, n_comp, x):
    import torch
    off, par, a, b, c, r = t
    s = torch.cuda.current_stream().cuda_stream
    return fn(off.numel() - 1, n_comp, off.data_ptr(), par.data_ptr(), a.data_ptr(), b.data_ptr(),
              c.data_ptr(), r.data_ptr(), x.data_ptr(), C.c_void_p(s))


def test_noalloc_matches_allocating_solve_on_two_calls_in_a_row():
    import torch
    torch.cuda.set_device(0)
    L = mm.load(build_if_missing=True)
    for seed, n_trees, max_n in ((11, 500, 40), (12, 60, 3000)):
        t = _device(_inputs(seed, n_trees, max_n))
        n = t[5].numel()
        x_ref = torch.empty_like(t[5])
        x_new = torch.full_like(t[5], float("nan"))
        assert _call(L.mm_hines_solve, t, n, x_ref) == mm.MM_OK
        assert _call(L.mm_hines_solve_noalloc, t, n, x_new) == mm.MM_OK
        np.testing.assert_allclose(x_new.cpu().numpy(), x_ref.cpu().numpy(), rtol=1e-12, atol=1e-14)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    L = mm.load(build_if_missing=True)
    t = _device(_inputs(13, 2, 4))
    x = torch.empty_like(t[5])
    assert _call(L.mm_hines_solve_noalloc, t, MAX_COMPS + 1, x) == mm.MM_EINVAL


def test_noalloc_rejects_bad_trees_and_leaves_no_stale_error():
    """A tree that breaks the parent rule, or whose offsets reach past n_comp,
    is rejected with MM_EINVAL through the no-allocation path; the next valid
    call on the same stream returns MM_OK (the shared status word starts at
    zero on every call) and matches the allocating solve."""
    import torch
    L = mm.load(build_if_missing=True)
    off, par, a, b, c, r = _inputs(14, 8, 30)
    bad_par = par.copy()
    bad_par[off[3]] = 0  # the root of tree 3 gets a parent
    t_bad = _device((off, bad_par, a, b, c, r))
    x = torch.empty_like(t_bad[5])
    assert _call(L.mm_hines_solve_noalloc, t_bad, t_bad[5].numel(), x) == mm.MM_EINVAL
    t = _device((off, par, a, b, c, r))
    assert _call(L.mm_hines_solve_noalloc, t, t[5].numel() - 1, x) == mm.MM_EINVAL  # last tree past n_comp
    x_ref = torch.empty_like(t[5])
    x_new = torch.full_like(t[5], float("nan"))
    assert _call(L.mm_hines_solve, t, t[5].numel(), x_ref) == mm.MM_OK
    assert _call(L.mm_hines_solve_noalloc, t, t[5].numel(), x_new) == mm.MM_OK
    np.testing.assert_allclose(x_new.cpu().numpy(), x_ref.cpu().numpy(), rtol=1e-12, atol=1e-14)
