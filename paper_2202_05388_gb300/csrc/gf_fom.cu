// Figure of merit of the current fields (Eq. 1: FOM = |E(r_m)|^2 at the monitor, summed over
// the wavelengths of a multi-wavelength problem and over the field components in 3-D).  The
// update kernels write the FOM after every step; this kernel gives it for a state no step has
// produced yet (right after a fill or a low-rank initialisation).
#include "gf_internal.cuh"

namespace gf {

// One thread sums components (outer) and wavelengths (inner) in the order the update's field
// kernel uses, so that the initial FOM and the per-step FOMs are computed alike.
__global__ void k_fom(FomArgs a, double* __restrict__ out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double f = 0.0;
  for (int q = 0; q < a.ncomp; ++q)
    for (int l = 0; l < a.nlam; ++l) f += abs2(a.E[l][a.mrow + q]);
  *out = f;
}

void launch_fom(const FomArgs& a, double* out, cudaStream_t st) { k_fom<<<1, 32, 0, st>>>(a, out); }

}  // namespace gf
