"""fea_row_ptr_from_counts_noalloc against the pattern builder's own row pointers.

Some callers cannot let a library allocate device memory (they reserve all of
it for their own pool, or run where an allocation would go through their
allocator or synchronize the device).  For them the library offers a row
pointer scan whose scratch is a fixed array compiled into the library.  This
test calls it through the C-ABI, twice in a row on the same inputs, and
requires bit-for-bit the row_ptr that fea_build_csr_pattern wrote.  It sits in
a file collected last so that a stop-at-first-failure run has already run
every other test.
"""
import ctypes

import pytest

from paper_1805_03949_gb300 import meshgen as mg
from tests.helpers import engine

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["hybrid6_scalar", "hex100_vector", "one_row"])
def test_noalloc_row_ptr_matches_pattern_builder(case):
    fea = engine()
    import torch
    if case == "hybrid6_scalar":
        mesh, ndof = mg.hybrid_cube(6, 3), 1
    elif case == "hex100_vector":
        mesh, ndof = mg.hex_cube(100, 0.2, 2), 3     # 3,090,903 rows: 755 tiles, ragged last tile
    else:
        mesh, ndof = mg.kuhn_tet_cube(0, 1, 1, 1), 1
    s = fea.System.from_mesh(mesh, ndof, with_cols=False)
    try:
        counts = (s.row_ptr[1:] - s.row_ptr[:-1]).to(torch.int32).contiguous()
        if case == "one_row":
            counts = counts[:1].contiguous()
        expect = s.row_ptr[:counts.numel() + 1]
        for _ in range(2):                           # the second call reuses the same scratch
            out = torch.full((counts.numel() + 1,), -7, dtype=torch.int64, device=counts.device)
            fea.fea_row_ptr_from_counts_noalloc(counts, out)
            torch.cuda.synchronize()
            assert torch.equal(out, expect)
    finally:
        s.close()


def test_noalloc_rejects_sizes_beyond_the_scratch():
    fea = engine()
    import torch
    counts = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(5, dtype=torch.int64, device="cuda")
    rc = fea.lib().fea_row_ptr_from_counts_noalloc(ctypes.c_void_p(counts.data_ptr()), 67_108_864 + 1,
                                                   ctypes.c_void_p(out.data_ptr()), None)
    assert rc == fea.FEA_ERR_UNSUPPORTED
    assert "scratch limit" in fea.fea_last_error()
    assert torch.count_nonzero(out).item() == 0      # nothing was written
