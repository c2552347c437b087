"""The partial-row decomposition of Sec. 3.1, on the oracle (CPU): the square
local matrices of an element partition, summed over the subdomains that hold
each node, give the globally assembled system."""
import numpy as np
import pytest

from paper_1805_03949_gb300 import meshgen as mg


def _csr(r, n):
    import scipy.sparse as sps
    return sps.csr_matrix((r["A"], r["col_idx"], r["row_ptr"]), shape=(n, n))


@pytest.mark.parametrize("name,parts", [("hex", 3), ("hybrid", 4), ("tet", 2)])
def test_local_matrices_sum_to_the_global_system(oracle, name, parts):
    import scipy.sparse as sps
    mesh = {"hex": lambda: mg.hex_cube(4, 0.2, 3), "hybrid": lambda: mg.hybrid_cube(3, 5),
            "tet": lambda: mg.kuhn_tet_cube(3)}[name]()
    d = 3
    ref = oracle.assemble(mesh, oracle.OP_ELASTICITY, tet_rule=1, poisson=0.3)
    Ag = _csr(ref, d * mesh.n_nodes)
    subs, mult = mg.partition_elements(mesh, parts)
    assert sum(s.n_elems for s, _ in subs) == mesh.n_elems
    assert (mult >= 1).all() and (mult > 1).any()        # every node held, some on interfaces
    total = sps.csr_matrix(Ag.shape)
    btot = np.zeros(d * mesh.n_nodes)
    for sub, glob in subs:
        r = oracle.assemble(sub, oracle.OP_ELASTICITY, tet_rule=1, poisson=0.3)
        P = sps.csr_matrix((np.ones(d * len(glob)),
                            (np.arange(d * len(glob)), (d * glob[:, None] + np.arange(d)).ravel())),
                           shape=(d * len(glob), d * mesh.n_nodes))
        total = total + P.T @ _csr(r, d * sub.n_nodes) @ P
        btot += P.T @ r["b"]
    scale = abs(Ag).max()
    assert abs(total - Ag).max() <= 1e-14 * scale
    np.testing.assert_allclose(btot, ref["b"], rtol=0, atol=1e-14 * np.abs(ref["b"]).max())
    # interface rows are partial in each subdomain: the node's row in one
    # subdomain alone differs from the global row exactly at shared nodes
    sub, glob = subs[0]
    r = oracle.assemble(sub, oracle.OP_ELASTICITY, tet_rule=1, poisson=0.3)
    loc = _csr(r, d * sub.n_nodes)
    shared = np.nonzero(mult[glob] > 1)[0]
    own = np.nonzero(mult[glob] == 1)[0]
    assert len(shared) and len(own)
    cols = (d * glob[:, None] + np.arange(d)).ravel()
    for i, complete in ((own[0], True), (shared[0], False)):
        row = np.zeros(d * mesh.n_nodes)
        row[cols] = loc[d * i].toarray().ravel()
        diff = np.abs(row - Ag[d * glob[i]].toarray().ravel()).max()
        assert (diff <= 1e-14 * scale) == complete, (i, complete, diff)
