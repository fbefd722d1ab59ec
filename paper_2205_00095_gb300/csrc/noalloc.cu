// Right-hand side without any device allocation: dgsrhd_rhs_noalloc.
//
// Some callers cannot allocate GPU memory at all: code that runs inside a host framework which
// owns every device allocation (a memory pool that forbids foreign cudaMalloc), code that runs
// where cudaMalloc would synchronise or fail (for example inside another library's callback or
// after the device memory has been reserved in full), or embedded users that must know their
// whole device footprint at load time.  For them this file keeps the scratch of one
// right-hand-side evaluation (volume term, face traces, face fluxes, counters) in a fixed
// array in device global memory that exists as soon as the library is loaded on a GPU, and
// offers one entry point that uses it instead of a context's buffers.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/dgsrhd.h"
#include "launch.h"
#include "params.h"

namespace {

// Capacity of the fixed scratch: 64 MiB of doubles on every GPU that loads the library, held
// until the process exits.
constexpr long long kScratchDoubles = (64LL << 20) / 8;

static __device__ __align__(256) double g_rhs_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  The symbol's host-side name is
// only a stand-in, so the address comes from cudaGetSymbolAddress with the device current.  It
// is looked up again on every call made outside stream capture (a device reset, or another
// context on the same device, loads the module at another address) and kept per device for
// calls made while `stream` is being captured, which reuse the address of the last call made
// outside capture on that device.
cudaError_t scratch_address(cudaStream_t stream, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (cap == cudaStreamCaptureStatusNone) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_rhs_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(ptr);
  } else if (!g_scratch_addr[dev]) {
    return cudaErrorStreamCaptureUnsupported;  // no address taken outside capture yet
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int32_t dgsrhd_rhs_noalloc(const dgsrhd_config* cfg, void* stream, const double* U,
                                      double* R, dgsrhd_stats* stats_out) {
  using namespace dgsrhd;
  if (!cfg || !U || !R || U == R) return DGSRHD_EINVAL;
  Params p;
  long long n_trace = 0, n_face_flux = 0;
  if (!params_from_config(cfg, &p, &n_trace, &n_face_flux)) return DGSRHD_EINVAL;
  const bool split = cfg->precision == DGSRHD_PREC_SPLIT;
  const long long n_state = 5 * p.E * p.Nn;
  // split precision: the per-element reference fluxes, FP32 head and tail in one double each
  const long long n_ref = split ? 5LL * p.dim * p.E : 0;
  const long long n_stats = (long long)kStatCount * 64;  // unsigned long long slots
  const long long need = n_state + n_trace + n_face_flux + n_ref + n_stats;
  if (need > kScratchDoubles) return DGSRHD_EINVAL;  // mesh too large for the fixed scratch

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* base = nullptr;
  if (scratch_address(s, &base) != cudaSuccess) return DGSRHD_ECUDA;
  double* Rvol = base;
  double* Tr = Rvol + n_state;
  double* Fs = Tr + n_trace;
  double* Fref = Fs + n_face_flux;
  unsigned long long* stats = reinterpret_cast<unsigned long long*>(Fref + n_ref);
  p.stats = stats;
  // the counters accumulate with atomics and must start at zero on every call
  if (cudaMemsetAsync(stats, 0, sizeof(unsigned long long) * n_stats, s) != cudaSuccess)
    return DGSRHD_ECUDA;

  StageArgs a{};
  a.p = &p;
  a.stream = s;
  a.U = U;
  a.Rvol = Rvol;
  a.Tr = Tr;
  a.Fs = Fs;
  a.Uout = R;
  a.mode = 0;
  // the split configuration runs the split kernels, as dgsrhd_rhs does
  a.split = split ? 1 : 0;
  a.Fref = split ? Fref : nullptr;
  const Op ops[3] = {Op::Volume, Op::Face, Op::Update};
  for (Op op : ops) {
    a.op = op;
    cudaError_t e;
    switch (p.dim) {
      case 1: e = dispatch_stage<1>(p.N, a); break;
      case 2: e = dispatch_stage<2>(p.N, a); break;
      default: e = dispatch_stage<3>(p.N, a); break;
    }
    if (e != cudaSuccess) return DGSRHD_ECUDA;
  }
  if (!stats_out) return DGSRHD_OK;

  unsigned long long h[kStatCount * 64];
  if (cudaMemcpyAsync(h, stats, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return DGSRHD_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return DGSRHD_ECUDA;
  unsigned long long v[kStatCount] = {0};
  for (int k = 0; k < kStatCount; ++k)
    for (int j = 0; j < 64; ++j) {
      const unsigned long long x = h[k * 64 + j];
      v[k] = (k == kStatItersMax) ? (x > v[k] ? x : v[k]) : v[k] + x;
    }
  stats_out->c2p_calls = p.E * p.Nn;
  stats_out->c2p_iters_total = (int64_t)v[kStatItersTotal];
  stats_out->c2p_iters_max = (int64_t)v[kStatItersMax];
  stats_out->c2p_nonconverged = (int64_t)v[kStatNonConv];
  stats_out->c2p_invalid_input = (int64_t)v[kStatInvalid];
  stats_out->face_guard_hits = (int64_t)v[kStatFaceGuard];
  stats_out->enforced_cells = 0;
  stats_out->mean_inadmissible_cells = 0;
  stats_out->limited_cells = 0;
  if (stats_out->c2p_invalid_input) return DGSRHD_EBADSTATE;
  if (stats_out->c2p_nonconverged) return DGSRHD_EC2P_NOCONV;
  return DGSRHD_OK;
}
