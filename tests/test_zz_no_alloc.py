"""The allocation-free Lindbladian application against the handle-based one.

lindbladian_apply_noalloc keeps its scratch in a fixed device array inside the library; it must
give the same L(X) as lindbladian_apply on consecutive calls (the second call reuses the scratch
the first one left behind), whatever ran before it in the process.
"""
import numpy as np
import pytest
import torch

import lindblad_inputs as gi

pytestmark = pytest.mark.gpu


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("n,d", [(48, 3), (131, 2)])
def test_noalloc_matches_handle_path_twice(n, d):
    import paper_2608_30860_b300 as B
    H, Ls = gi.random_lindbladian(n, d=d, seed=n)
    Hd, Ld = _cuda(H), _cuda(np.stack(Ls))
    h = B.lindblad_setup(Hd, Ld)
    for seed in (1, 2):
        X = _cuda(gi.random_operator(n, seed=seed))
        ref = B.lindbladian_apply(h, X)
        got = B.lindbladian_apply_noalloc(Hd, Ld, X)
        torch.cuda.synchronize()
        err = float((got - ref).abs().max() / ref.abs().max())
        assert err < 1e-13, err
    B.lindblad_destroy(h)


def test_noalloc_refuses_oversize():
    import paper_2608_30860_b300 as B
    n = 513
    H = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    L = torch.zeros((1, n, n), dtype=torch.complex128, device="cuda")
    with pytest.raises(B.LindbladError):
        B.lindbladian_apply_noalloc(H, L, H)
