// gf_fill_g0_static: the background fill of gf_fill_g0 for callers that cannot allocate
// device memory.  The paper has no counterpart; this is a deployment convenience.
//
// gf_fill_g0 needs scratch space for its Toeplitz table of Hankel-function values (2N
// complex128 entries) and takes it from a caller workspace.  Some callers cannot provide one:
// code that runs inside a host application which owns every device allocation and hands out
// no scratch (plug-ins, embedded solvers), or a latency-critical loop that must not call
// cudaMalloc because it can synchronise the device.  This entry point keeps the table in a
// fixed array in device global memory that is part of the library image instead.
//
// Limits and sharing rules:
//   * the array holds kStaticTableEntries = 2^18 complex128 entries (4 MiB), so the design
//     may have at most 2^17 = 131072 pixels; larger grids are rejected with GF_EINVAL;
//   * every GPU that loads the library holds these 4 MiB until the process exits;
//   * all calls on a device share the one array and it keeps the last call's contents; each
//     call writes every table entry it reads, so nothing has to start at zero;
//   * calls that overlap on the GPU (for example on two streams) race on the array and must
//     be ordered by the caller;
//   * every call looks up the array's device address with cudaGetSymbolAddress, with the
//     handle's device current, and checks the result; the first call on a device also loads
//     the library's device code there, so make that first call before any stream capture.
//     Looking the address up per call (a host-side table lookup once the code is loaded) keeps
//     it right after the device's context has been torn down and created again, where a
//     cached address would point into memory that no longer belongs to the array.
#include "gf_internal.cuh"

namespace gf {

constexpr int64_t kStaticTableEntries = int64_t(1) << 18;

static __device__ __align__(256) cplx g_static_table[kStaticTableEntries];

// Device address of g_static_table on the current device.
static cplx* static_table_address(cudaError_t* err) {
  void* p = nullptr;
  *err = cudaGetSymbolAddress(&p, g_static_table);
  return *err == cudaSuccess ? reinterpret_cast<cplx*>(p) : nullptr;
}

}  // namespace gf

extern "C" gf_status gf_fill_g0_static(gf_handle* h, const gf_problem* prob, int32_t dtype, void* stream) {
  if (!h) return GF_EINVAL;
  gf_status s = gf::api_check_problem(h, prob, dtype);
  if (s) return s;
  const int64_t N = (int64_t)prob->geom.nx * prob->geom.ny;
  if (2 * N > gf::kStaticTableEntries)
    return gf::api_fail_msg(h, GF_EINVAL,
                            "gf_fill_g0_static supports at most 131072 pixels (its fixed 4 MiB table "
                            "holds 2N entries); use gf_fill_g0 with a workspace for larger grids");
  if ((s = gf::api_bind_device(h))) return s;
  cudaError_t e;
  gf::cplx* table = gf::static_table_address(&e);
  if (!table) {
    cudaGetLastError();
    return gf::api_fail_msg(h, GF_ECUDA, cudaGetErrorString(e));
  }
  cudaStream_t st = (cudaStream_t)stream;
  gf::launch_fill_table(prob->geom, table, st);
  gf::launch_fill_expand(prob->geom, dtype, prob->G, prob->ldg, table, reinterpret_cast<gf::cplx*>(prob->E), st);
  gf::launch_bands(prob->geom, dtype, prob->G, prob->ldg, reinterpret_cast<gf::cplx*>(prob->bands), st);
  return gf::api_cuda_check(h, "gf_fill_g0_static launch");
}
