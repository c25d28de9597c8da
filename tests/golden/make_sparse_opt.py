"""Writes tests/golden/zipf_csr_opt.txt: the reference optimum of the seeded
Zipf term-document matrices (no planted spectrum, so no closed form).

opt = ||X||_F^2 - sum_{j<=k} lambda_j(X X^T), the eigenvalues from ARPACK
Lanczos (oracle.top_eigs_lanczos), cross-checked by the oracle's plain
subspace iteration (Algorithm 1 on A with exact products, then Algorithm 2):
the two must agree to 1e-8 relative on opt.  Calls only oracle/ and the input
generator.  Usage: python tests/golden/make_sparse_opt.py [name ...]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import lra_inputs as L  # noqa: E402
from oracle import lra_oracle as O  # noqa: E402


def main(names):
    import scipy.sparse as sp
    out = os.path.join(HERE, "zipf_csr_opt.txt")
    lines = []
    for name in names:
        wl = L.WORKLOADS[name]
        t0 = time.time()
        rowptr, colidx, val = L.zipf_csr(wl.d, wl.n, wl.seed)
        Xt = sp.csr_matrix((val, colidx, rowptr), shape=(wl.d, wl.n)).T.tocsr().astype(np.float64)
        fro2 = O.colnorms(Xt)[1]
        lam = O.top_eigs_lanczos(Xt, wl.p + 1)
        opt = fro2 - float(np.sum(lam[:wl.k]))
        rho = O.plain_subspace_iteration(Xt, wl.k, wl.p, 300)
        opt_si = fro2 - float(np.sum(rho[:wl.k]))
        agree = abs(opt_si - opt) / opt
        print(f"{name}: fro2 {fro2:.12g} opt {opt:.12g} (subspace iteration {opt_si:.12g}, rel {agree:.2e}) "
              f"lambda_1..{wl.p + 1} {np.array2string(lam, precision=8)} [{time.time() - t0:.0f} s]", flush=True)
        assert agree < 1e-8, agree
        lines.append(f"{name} k={wl.k} fro2={fro2:.15g} opt={opt:.15g} "
                     f"lambda_k={lam[wl.k - 1]:.15g} lambda_k1={lam[wl.k]:.15g} lambda_p1={lam[wl.p]:.15g}")
    with open(out, "w") as f:
        f.write("# Reference optima of the seeded Zipf CSR workloads: ||X||_F^2 - sum of the top-k\n")
        f.write("# eigenvalues of X X^T (ARPACK Lanczos, FP64), cross-checked by 300 steps of plain\n")
        f.write("# subspace iteration with Rayleigh-Ritz (Algorithms 1-2 on A).\n")
        f.write("# Written by tests/golden/make_sparse_opt.py from oracle/ only.\n")
        for ln in lines:
            f.write(ln + "\n")


if __name__ == "__main__":
    main(sys.argv[1:] or ["zipf_csr_2000x20000", "zipf_csr_50000x500000"])
