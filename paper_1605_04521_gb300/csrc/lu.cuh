// Types shared by the LU kernels (lu.cu) and the tensor-core trailing update (lu_tc.cu).
#pragma once

#include <climits>

#include "dev.cuh"

namespace oras {

// Rectangular set of output tiles [i0, i1) x [j0, j1); an end of INT_MAX means the subdomain's
// tile count.
struct Region { int i0, i1, j0, j1; };
struct UpdArgs {
  int kk0, kk1;             // contraction over tile columns [kk0, kk1)
  int nreg;
  Region reg[2];
};

// Clip a region to a subdomain with nts tile rows/columns.
__host__ __device__ __forceinline__ void region_clip(const Region& r, int64_t nts, int64_t& i0, int64_t& i1,
                                                     int64_t& j0, int64_t& j1) {
  i0 = r.i0;
  j0 = r.j0;
  i1 = r.i1 == INT_MAX ? nts : (r.i1 < nts ? r.i1 : nts);
  j1 = r.j1 == INT_MAX ? nts : (r.j1 < nts ? r.j1 : nts);
  if (i1 < i0) i1 = i0;
  if (j1 < j0) j1 = j0;
}

// tensor-core trailing update (lu_tc.cu): returns false when it cannot run (then the caller
// uses the CUDA-core kernel)
bool tc_update_available(oras_handle* h);
int launch_update_tc(oras_handle* h, const UpdArgs& u, int max_nts, int cls);
// tile solves of step k with the inverted diagonal blocks in the scratch slots: the tiles below
// the diagonal (when lower) and row k's tiles in columns [ju0, ju1)
int launch_trsm_tc(oras_handle* h, int k, int max_nts, bool lower, int ju0, int ju1, int l_slot);

}  // namespace oras
