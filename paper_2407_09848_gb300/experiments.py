"""Experiments of the paper reproduced on the GPU path.

smoother_only: the remark of Sec. 2.3 -- PCG iteration counts (tol 1e-5,
b = A 1) when the preconditioner is one application of the optimised
1st-kind (Algorithm 1) or 4th-kind (Eq. polsmootheropt) polynomial smoother
alone, on A = Q D Q^T with equispaced, boundary-clustered and gapped spectra,
for several sizes and degrees.  The paper shows these counts only as images.

CLI:  python -m paper_2407_09848_gb300.experiments smoother_only
"""
from __future__ import annotations

import json
import sys

import numpy as np

from . import problems as pr


def smoother_only(sizes=(128, 256, 512, 1024), degrees=(1, 2, 3, 4, 5, 6, 8, 10, 12),
                  spectra=("equispaced", "boundary", "gap"), rtol=1e-5):
    import torch
    from .amgps import Solver
    out = []
    for spec in spectra:
        for N in sizes:
            A, b = pr.spectral_test_matrix(N, spec)
            As, Ps = pr.single_aggregate_hierarchy(A)
            S = Solver().load(As, Ps)
            bd = torch.from_numpy(b).cuda()
            x = torch.empty_like(bd)
            for k in degrees:
                row = {"spectrum": spec, "N": N, "degree": k}
                for kind in ("cheb1_opt", "cheb4_opt"):
                    it, rel = S.pcg_smoother(kind, k, bd, x, rtol=rtol, maxit=20000,
                                             raise_on_noconv=False)
                    row[kind] = it
                out.append(row)
            S.close()
    return out


def main(argv):
    if len(argv) < 1 or argv[0] != "smoother_only":
        print(__doc__)
        return 2
    rows = smoother_only()
    print(json.dumps(rows))
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
