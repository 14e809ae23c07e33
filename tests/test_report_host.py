"""Host-side pin of the CSR count used in the storage report."""
import numpy as np
import scipy.sparse as sp

from paper_1811_06797_gb300.report import csr_nnz


def test_csr_nnz_is_the_kronecker_band_pattern():
    for n, p in (((5, 7, 4), (1, 2, 3)), ((9, 9, 9), (2, 2, 2)), ((3, 2, 6), (3, 3, 1))):
        mats = []
        for nd, pd in zip(n, p):
            ks = [k for k in range(-pd, pd + 1) if abs(k) < nd]
            mats.append(sp.diags([np.ones(nd - abs(k)) for k in ks], ks, shape=(nd, nd)))
        A = sp.kron(mats[0], sp.kron(mats[1], mats[2]))
        assert csr_nnz(n, p) == sp.csr_matrix(A).count_nonzero()
