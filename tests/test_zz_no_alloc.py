"""The allocation-free operator apply (ocg_apply_A_f32_noalloc).

Some callers cannot allocate device memory when they call into the solver: a host
framework that owns all device memory through its own pool, a loop with a hard latency
budget that may not block in cudaMalloc, or a process running under an external memory
cap.  For them the library offers one operator apply whose work vectors sit in a fixed
array compiled into the library.  This file checks, through the C ABI, that it returns
what the regular apply (ocg_apply_A, FP32) returns, on two calls in a row, and that it
refuses trees larger than its fixed array.  It is collected last so a stop at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2604_18886_b300 import _lib as L
from paper_2604_18886_b300 import problems as P
from paper_2604_18886_b300 import solver as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _apply_noalloc(h, x):
    y = torch.empty_like(x)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.check(L.lib().ocg_apply_A_f32_noalloc(h.handle, L.ptr(x), L.ptr(y), st))
    torch.cuda.synchronize()
    return y


@pytest.mark.parametrize("coef", ["f32", "f64"])
def test_noalloc_apply_matches_regular_apply_twice(coef):
    p = P.cut_cell(16, 2)
    tree = S.Octree(p.desc)
    beta = P.face_beta(p, tree.faces())
    hier = S.Hierarchy(tree, beta, p.bc, S.mg_params(coef=coef))
    rng = np.random.default_rng(17)
    for _ in range(2):
        x = torch.from_numpy(rng.standard_normal(tree.n_leaves).astype(np.float32)).cuda()
        ref = hier.apply_A(x)
        y = _apply_noalloc(hier, x)
        err = (y.double() - ref.double()).abs().max().item() / ref.double().abs().max().item()
        assert err <= 1e-6


def test_noalloc_apply_rejects_trees_above_the_limit():
    p = P.uniform(128)                       # 2,097,152 tree cells > 2^20
    tree = S.Octree(p.desc)
    assert tree.n_tree > L.OCG_NOALLOC_MAX_CELLS
    hier = S.Hierarchy(tree, np.ones(tree.n_faces, np.float32), p.bc)
    x = torch.zeros(tree.n_leaves, dtype=torch.float32, device="cuda")
    with pytest.raises(L.OcgError) as e:
        _apply_noalloc(hier, x)
    assert e.value.code == L.OCG_EINVAL
