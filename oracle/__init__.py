"""CPU oracle for the sparse product C = A.B and its k-slice merge.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this package; the GPU library never imports,
links or calls it, and it shares no code with the GPU library (the only common
module is the seeded input generator, which holds none of the product's
arithmetic).  Operands are any objects with ``nrows, ncols, rowptr, col, val``.

Parts and the passages they follow:

* ``spgemm``        -- Gustavson with a dense sparse accumulator (Alg. 1, Sec. 3),
                       plain C in ``spa_oracle.c``.  Pinned by the tests in
                       ``tests/test_oracle.py`` (dense matmul, transpose and
                       identity identities, K_n closed form, AMG closed form,
                       permutation equivariance, nnz(C) <= flops).
* ``sum_partials``  -- the multiway merge's result, C = sum_s C_s (Sec. 4.3).
                       Pinned by merge(slices) == unsplit product.
* ``kslice``        -- the split of the inner dimension into c contiguous
                       ranges (Sec. 4.1 split distribution, Alg. 2).
* ``transpose``     -- plain CSR transpose (Alg. 2 transposes B locally).
* ``row_flops``     -- flops(A,B) per row (Sec. 2 "Notation").
* ``mlp``           -- float64 reference of the row-size predictor (not in the
                       paper; see ``oracle/mlp.py``).
* ``mcl``           -- prune + column renormalisation of a Markov matrix
                       (Markov clustering expansion, Sec. 5.3).
* ``spgemm`` semirings "min_plus" / "min_select2nd" and ``mask`` -- the
                       operations MIS-2 aggregation is built from (Alg. 3):
                       pinned by brute force, a path-graph closed form, the
                       identity and a row-selection reduction; the mask by set
                       identities (full mask, complement partition).
"""
from .core import (OCSR, spgemm, sum_partials, kslice_bounds, kslice, transpose, row_flops,
                   abs_bound, mcl_prune_renorm, lib_path, build, num_threads, mask)

__all__ = ["OCSR", "spgemm", "sum_partials", "kslice_bounds", "kslice", "transpose", "mask",
           "row_flops", "abs_bound", "mcl_prune_renorm", "lib_path", "build", "num_threads"]
