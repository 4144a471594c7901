"""The allocation-free preconditioner apply gives the regular apply's result.

oras_precond_noalloc exists for callers that cannot allocate device memory during a call (a
pool allocator owns all of the device memory, or cudaMalloc's device synchronisation would
stall other requests in flight).  It keeps its local vectors in a fixed device array inside the
library.  This file is collected last on purpose: it must pass both alone in a fresh process and
after every other GPU test.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_noalloc_apply_matches_regular_apply_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_04521_gb300 import build
    build.build()
    from paper_1605_04521_gb300 import oras as O
    w = synth.small(n=4, r=2, nsub=8, overlap=1)
    xyz, tets = w.mesh()
    eps, mu = w.materials(xyz, tets)
    # ORAS with FP32 and FP64 factors, and OAS (no partition of unity: the overlapping
    # contributions are summed into z, which the call clears first)
    for bits, weights in ((32, O.ORAS_WEIGHTS_POU), (64, O.ORAS_WEIGHTS_POU), (32, O.ORAS_WEIGHTS_NONE)):
        h = O.oras_setup(xyz, tets, eps, mu, w.k0, w.r, w.nsub, w.overlap, factor_bits=bits, weights=weights)
        try:
            n = O.oras_ndof(h)
            rng = np.random.default_rng(bits)
            for call in range(2):            # two calls in a row share the fixed array
                k = 1 + call
                v = rng.normal(size=(k, n)) + 1j * rng.normal(size=(k, n))   # column-major N x k
                ref = O.oras_precond(h, v.T.copy(), k=k)
                ref = ref.reshape(n, k) if k > 1 else ref[:, None]
                vd = torch.from_numpy(v).cuda()
                zd = torch.full_like(vd, complex(np.nan, np.nan))
                O.oras_precond_noalloc(h, vd, zd, k)
                torch.cuda.synchronize()
                got = zd.cpu().numpy().T
                err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
                # the regular apply may give the largest subdomains four CTAs (this one always
                # takes two), which sums each strip's products in another order: with FP32
                # factors the two agree to FP32 rounding, with FP64 factors to FP64 rounding
                assert err <= (1e-5 if bits == 32 else 1e-12), (bits, weights, call, err)
        finally:
            O.oras_destroy(h)
