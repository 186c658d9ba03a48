// Diagnostic of the bounded waits the tensor-core kernels rely on: a kernel waits on an
// mbarrier that nothing signals, with the same abortable wait and a caller-given limit, and
// reports GF_ETIMEOUT through the device status word -- the path a stalled pipeline takes,
// exercised without any GPU fault (the context stays usable afterwards).
#include "gf_internal.cuh"
#include "gf_tc.cuh"

namespace gf {

__global__ void k_selftest_timeout(uint64_t timeout_ns, int32_t* __restrict__ status) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    abort_flag = 0;
    tc::fence_mbar_init();
  }
  __syncthreads();
  bool ok = true;
  if (threadIdx.x == 0) ok = tc::mbar_wait_or_abort(&bar, 0, &abort_flag, timeout_ns);   // nobody arrives
  __syncthreads();
  if (threadIdx.x == 0) *status = (!ok && abort_flag) ? GF_ETIMEOUT : GF_OK;
}

}  // namespace gf

extern "C" gf_status gf_selftest_timeout(gf_handle* h, int64_t timeout_ns, int32_t* status, void* stream) {
  if (!h) return GF_EINVAL;
  if (!status || timeout_ns < 1000 || timeout_ns > 2000000000ll)
    return gf::api_fail_msg(h, GF_EINVAL, "status must be non-NULL and timeout_ns in [1 us, 2 s]");
  gf_status s = gf::api_bind_device(h);
  if (s) return s;
  gf::k_selftest_timeout<<<1, 32, 0, (cudaStream_t)stream>>>((uint64_t)timeout_ns, status);
  return gf::api_cuda_check(h, "gf_selftest_timeout launch");
}

extern "C" size_t gf_select_selftest_bytes(void) { return gf::topk_selftest_bytes(); }

extern "C" gf_status gf_select_selftest_timeout(gf_handle* h, int64_t timeout_ns, void* ws, size_t ws_bytes,
                                                int32_t* status, void* stream) {
  if (!h) return GF_EINVAL;
  if (!status || !ws || ((uintptr_t)ws & 255u) || timeout_ns < 1000 || timeout_ns > 2000000000ll)
    return gf::api_fail_msg(h, GF_EINVAL,
                            "status and a 256-byte aligned ws must be given and timeout_ns lie in [1 us, 2 s]");
  if (ws_bytes < gf::topk_selftest_bytes())
    return gf::api_fail_msg(h, GF_ENOMEM, "ws is smaller than gf_select_selftest_bytes()");
  gf_status s = gf::api_bind_device(h);
  if (s) return s;
  if (!gf::launch_topk_selftest(ws, (uint64_t)timeout_ns, status, (cudaStream_t)stream))
    return gf::api_fail_msg(h, GF_ECUDA, "the device cannot launch the one-launch top-k (cooperative launch)");
  return gf::api_cuda_check(h, "gf_select_selftest_timeout launch");
}
