// Single-graph blocked Floyd-Warshall: host driver and C ABI (include/apsp.h).
//
// Per call: validate, pick the arithmetic (fp32, or exact 16-bit when every
// path length fits), lay D/P out in a working layout whose order is a multiple
// of 128, then run R = n_pad/BS block rounds (Section 4.1 of arXiv 1811.01201),
// each as four stream-ordered launches: phase 1 (diagonal block), phase 2 (its
// row and column blocks), the panel pack, phase 3 (all remaining blocks).
// Kernel boundaries are the barriers between the phases; the kernels are
// launched as programmatic dependents, so each is scheduled while its
// predecessor runs and waits on the device for it to finish.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <vector>

#include "../../include/apsp.h"
#include "apsp_internal.h"
#include "fw_aux.cuh"
#include "fw_minplus_f32.cuh"
#include "fw_minplus_u16.cuh"
#include "fw_seq.cuh"

namespace apsp {

int current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return (dev >= 0 && dev < kMaxDevices) ? dev : -1;
}

int sm_count() {
  static std::atomic<int> cache[kMaxDevices];
  const int dev = current_device();
  if (dev < 0) return 152;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v <= 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 152;
    }
    cache[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

static int elementwise_grid(size_t work) {
  const size_t per = 256;
  size_t g = (work + per - 1) / per;
  return (int)std::max<size_t>(1, std::min<size_t>(g, (size_t)sm_count() * 16));
}

// ---------------------------------------------------------------- phase timing

// Optional per-phase device timing (APSP_FLAG_TIME_PHASES): an event after
// every phase launch; interval i is charged to the phase that ended it.
struct PhaseTimer {
  cudaStream_t s = nullptr;
  std::vector<cudaEvent_t> ev;
  std::vector<int> tag;
  int launches[3] = {0, 0, 0};
  int other = 0;  // launches outside the three phases' own kernels (panel packing)
  bool on = false;
  void mark(int phase) {
    if (phase >= 0) ++launches[phase];
    if (!on) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, s);
    ev.push_back(e);
    tag.push_back(phase);
  }
  void finish(float ms[3]) {
    ms[0] = ms[1] = ms[2] = 0.f;
    if (on && !ev.empty()) {
      cudaEventSynchronize(ev.back());
      for (size_t i = 1; i < ev.size(); ++i) {
        float t = 0.f;
        if (tag[i] >= 0 && cudaEventElapsedTime(&t, ev[i - 1], ev[i]) == cudaSuccess) ms[tag[i]] += t;
      }
    }
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    ev.clear();
    tag.clear();
  }
};

// ---------------------------------------------------------------- launch tables

// Launch with programmatic stream serialization: the kernel may be scheduled
// while its predecessor in the stream still runs; it waits for it in
// pdl_prologue (every round kernel starts with that).
template <typename... KArgs, typename... Args>
static cudaError_t launch_dependent(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                                    cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// First-wave stagger of the fp32 phase-3 launch (cycles; see the kernel).
constexpr int kStaggerCycles = 6000;
// Limit of a phase-3 CTA's wait for its panel slices (they arrive in
// microseconds), and the short limit used with APSP_FLAG_TEST_PANEL_TIMEOUT.
constexpr unsigned long long kPanelWaitNs = 2000000000ull;
constexpr unsigned long long kPanelWaitTestNs = 20000000ull;

template <class T, int BS>
static cudaError_t launch_rounds_bs(typename T::store_t* D, int32_t* P, int n_pad, cudaStream_t s, PhaseTimer& tm,
                                    RoundMax* rm, int graph_int, float* pan, void* pdiag, int flags) {
  const int R = n_pad / BS;
  const int nT = n_pad / kTile;
  const size_t ld = (size_t)n_pad;
  constexpr size_t sm1 = phase1_smem_bytes<T, BS>();
  constexpr size_t sm2 = phase2_smem_bytes<T, BS>();
  constexpr size_t sm3 = std::is_same<T, F32T>::value ? minplus_f32_smem_bytes<BS>() : minplus_u16_smem_bytes<BS>();
  constexpr size_t sm3r = minplus_f32_real_smem_bytes<BS>();
  // Function attributes belong to the device that was current when they were set.
  static std::once_flag once[kMaxDevices];
  static cudaError_t attr_errs[kMaxDevices];
  const int dev = current_device();
  if (dev < 0) return cudaErrorInvalidDevice;
  cudaError_t& attr_err = attr_errs[dev];
  std::call_once(once[dev], [&attr_err] {
    cudaError_t e1 = cudaFuncSetAttribute(fw_phase2_kernel<T, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
    const cudaError_t e0 =
        cudaFuncSetAttribute(fw_phase1_kernel<T, BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if (e1 == cudaSuccess) e1 = e0;
    cudaError_t e2, e3 = cudaSuccess;
    if constexpr (std::is_same<T, F32T>::value) {
      e2 = cudaFuncSetAttribute(fw_phase3_f32_kernel<BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3);
      e3 = cudaFuncSetAttribute(fw_phase3_f32_real_kernel<BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3r);
    } else {
      e2 = cudaFuncSetAttribute(fw_phase3_u16_kernel<BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3);
    }
    attr_err = e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3);
  });
  if (attr_err != cudaSuccess) return attr_err;
  const int sms = sm_count();
  // packed panel slices: nT A slices, then nT B slices
  float* Apk = pan;
  float* Bpk = pan + (size_t)nT * panel_slice_floats<BS>();
  const bool test_timeout = (flags & APSP_FLAG_TEST_PANEL_TIMEOUT) != 0;
  const unsigned long long wait_ns = test_timeout ? kPanelWaitTestNs : kPanelWaitNs;
  tm.mark(-1);
  using reg_t = typename T::reg_t;
  reg_t* pk = static_cast<reg_t*>(pdiag);
  cudaError_t err = cudaSuccess;
  auto keep = [&err](cudaError_t e) {
    if (err == cudaSuccess) err = e;
  };
  for (int r = 0; r < R && err == cudaSuccess; ++r) {
    keep(launch_dependent(fw_phase1_kernel<T, BS>, 1, SeqShape<BS>::NT, sm1, s, D, P, ld, r, rm, pk));
    tm.mark(0);
    if (R > 1) {
      keep(launch_dependent(fw_phase2_kernel<T, BS>, 2 * (R - 1), LineShape<BS>::NT, sm2, s, D, P, ld, r, R, rm,
                       static_cast<const reg_t*>(pk), wait_ns, (int)test_timeout, graph_int));
      tm.mark(1);
      if constexpr (std::is_same<T, F32T>::value) {
        if (graph_int) {
          keep(launch_dependent(fw_pack_panels_f32_kernel<BS>, 2 * nT, 256, 0, s, static_cast<const float*>(D), ld,
                                nT, r, static_cast<const RoundMax*>(rm), graph_int, Apk, Bpk));
          ++tm.other;
          keep(launch_dependent(fw_phase3_f32_kernel<BS>, nT * nT, 256, sm3, s, D, P, ld, nT, r, rm, graph_int,
                                static_cast<const float*>(Apk),
                                static_cast<const float*>(Bpk), kStaggerCycles, sms, wait_ns, (int)test_timeout));
        } else {
          // real-valued weights: B slices 64 columns wide, tiles of 128 x 64
          const int nTc = nT * (kTile / kRealCols);
          keep(launch_dependent(fw_pack_panels_f32_kernel<BS, kRealCols>, nT + nTc, 256, 0, s,
                                static_cast<const float*>(D), ld, nT, r, static_cast<const RoundMax*>(rm), 0, Apk,
                                Bpk));
          ++tm.other;
          keep(launch_dependent(fw_phase3_f32_real_kernel<BS>, nT * nTc, 256, sm3r, s, D, P, ld, nT, r, rm,
                                static_cast<const float*>(Apk), static_cast<const float*>(Bpk), kStaggerCycles, sms,
                                wait_ns, (int)test_timeout));
        }
      } else {
        uint32_t* Apk16 = reinterpret_cast<uint32_t*>(pan);
        uint32_t* Bpk16 = Apk16 + (size_t)nT * u16_slice_a_words<BS>();
        keep(launch_dependent(fw_pack_panels_u16_kernel<BS>, 2 * nT, 256, 0, s, static_cast<const uint16_t*>(D), ld, nT,
                              r, static_cast<const RoundMax*>(rm), Apk16, Bpk16));
        ++tm.other;
        keep(launch_dependent(fw_phase3_u16_kernel<BS>, nT * nT, 256, sm3, s, D, P, ld, nT, r, rm,
                         static_cast<const uint32_t*>(Apk16),
                         static_cast<const uint32_t*>(Bpk16), kStaggerCycles, sms, wait_ns, (int)test_timeout));
      }
      tm.mark(2);
    }
  }
  if (err != cudaSuccess) return err;
  return cudaGetLastError();
}

template <class T>
static cudaError_t launch_rounds(typename T::store_t* D, int32_t* P, int n_pad, int bs, cudaStream_t s,
                                 PhaseTimer& tm, RoundMax* rm, int graph_int, float* pan, void* pdiag, int flags) {
  switch (bs) {
    case 32: return launch_rounds_bs<T, 32>(D, P, n_pad, s, tm, rm, graph_int, pan, pdiag, flags);
    case 64: return launch_rounds_bs<T, 64>(D, P, n_pad, s, tm, rm, graph_int, pan, pdiag, flags);
    case 128: return launch_rounds_bs<T, 128>(D, P, n_pad, s, tm, rm, graph_int, pan, pdiag, flags);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------- planning

struct Plan {
  int n = 0, n_pad = 0, bs = 0, dtype = 0;
  bool in_place = false;
  size_t ws_stats = 0, ws_d = 0, ws_p = 0, ws_pan = 0, ws_diag = 0, ws_total = 0;  // byte offsets / total
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// Workspace layout for a given arithmetic and block size:
// [stats + round maxima][D work][P work][packed panel slices][packed diagonal block].
constexpr size_t kRoundMaxOffset = 64;  // RoundMax inside the 256-byte head
static size_t packed_panel_bytes(int n_pad, int bs, int dtype) {
  const size_t nT = (size_t)(n_pad / kTile);
  if (dtype == APSP_DTYPE_U16X2) return nT * (size_t)bs * (kSstA16 + kSstB16) * sizeof(uint32_t);
  // A slices plus B slices 128 columns wide (integer weights) or 64 wide (real weights)
  const size_t a = nT * (size_t)(bs / 2) * kS2;
  const size_t b = std::max(nT * (size_t)(bs / 2) * kS2, 2 * nT * (size_t)(bs / 2) * kRealSB);
  return (a + b) * sizeof(float);
}
static void layout(Plan& pl, bool p_in_place) {
  const size_t np2 = (size_t)pl.n_pad * pl.n_pad;
  size_t off = 0;
  pl.ws_stats = off;
  static_assert(sizeof(WeightStats) <= kRoundMaxOffset, "stats overlap the round maxima");
  off = align256(off + kRoundMaxOffset + sizeof(RoundMax));
  pl.ws_d = off;
  if (pl.dtype == APSP_DTYPE_U16X2) off = align256(off + np2 * sizeof(uint16_t));
  else if (!pl.in_place) off = align256(off + np2 * sizeof(float));
  pl.ws_p = off;
  if (!p_in_place) off = align256(off + np2 * sizeof(int32_t));
  pl.ws_pan = off;
  off = align256(off + packed_panel_bytes(pl.n_pad, pl.bs, pl.dtype));
  pl.ws_diag = off;
  off = align256(off + 2 * (size_t)pl.bs * (pl.bs + 4) * sizeof(uint32_t));
  pl.ws_total = off;
}

int padded_order(int n) { return ((n + kTile - 1) / kTile) * kTile; }

size_t fw_fault_word_offset() { return kRoundMaxOffset + offsetof(RoundMax, fault); }

bool u16_eligible(bool all_integer, bool complete, float max_w, int n) {
  if (!all_integer) return false;
  // every simple path, at most n-1 edges, stays below INF = 65535
  if ((double)max_w * (double)(n - 1) < 65535.0) return true;
  // with every edge present, D[i][j] never exceeds W[i][j] <= max_w, so every stored value
  // stays below 65535 and a saturated candidate never wins
  return complete && max_w < 65535.0f;
}

}  // namespace apsp

using namespace apsp;

// ---------------------------------------------------------------- ABI

extern "C" int apsp_default_bs(int n) {
  // measured on one GB300 (integer weights): BS = 64 is faster from n = 1024 up
  // (n = 1024: 2.2 vs 1.8 TFLOPS, n = 2048: 7.9 vs 6.4)
  if (n <= 512) return 32;
  return 64;
}

namespace apsp {
// Default block size once the arithmetic is known: the 16-bit path, whose hot
// loop is twice as fast, gains from fewer rounds on large n (n = 32768: 61.2
// vs 58.3 TFLOPS at BS = 128 and 64; equal at 16384; BS = 64 ahead below).
int default_bs_for(int n, int dtype) {
  if (dtype == APSP_DTYPE_U16X2 && n > 16384) return 128;
  return apsp_default_bs(n);
}
}  // namespace apsp

extern "C" const char* apsp_status_str(apsp_status s) {
  switch (s) {
    case APSP_OK: return "ok";
    case APSP_EINVAL: return "invalid argument";
    case APSP_ENOMEM: return "out of memory";
    case APSP_ECUDA: return "CUDA error";
    case APSP_ETIMEOUT: return "timed out";
    case APSP_EBUSY: return "busy / not ready";
    case APSP_ECANCELLED: return "cancelled";
    case APSP_ENOTFOUND: return "not found";
  }
  return "unknown status";
}

static apsp_options default_options() {
  apsp_options o;
  std::memset(&o, 0, sizeof(o));
  o.bs = 0;
  o.dtype = APSP_DTYPE_AUTO;
  o.validate = 1;
  return o;
}

static bool valid_bs(int bs) { return bs == 32 || bs == 64 || bs == 128; }

namespace apsp {

// Workspace plan of fw_exec: the solve runs in place in the caller's D (fp32
// path) and P only when n is a multiple of 128 and that matrix starts on a
// 16-byte boundary (the vector loads and bulk copies need it); otherwise the
// workspace also holds a padded working copy.
static Plan plan_for(int n, int bs, int dtype, const void* D, const void* P, bool* p_in_place) {
  Plan pl;
  pl.n = n;
  pl.n_pad = padded_order(n);
  pl.bs = bs;
  pl.dtype = dtype;
  const bool pad = pl.n_pad != n;
  *p_in_place = !pad && aligned16(P);
  pl.in_place = (dtype == APSP_DTYPE_F32) && !pad && aligned16(D);
  layout(pl, *p_in_place);
  return pl;
}

size_t fw_exec_workspace(int n, int bs, int dtype, const void* D, const void* P) {
  bool p_in_place = false;
  return plan_for(n, bs, dtype, D, P, &p_in_place).ws_total;
}

size_t fw_workspace_need(int n, const apsp_options* opt, const void* D, const void* P) {
  apsp_options o = opt ? *opt : default_options();
  if (n < 1 || n > 65536) return 0;
  if (o.bs != 0 && !valid_bs(o.bs)) return 0;
  size_t need = 0;
  if (o.dtype != APSP_DTYPE_U16X2)
    need = fw_exec_workspace(n, o.bs ? o.bs : default_bs_for(n, APSP_DTYPE_F32), APSP_DTYPE_F32, D, P);
  if (o.dtype != APSP_DTYPE_F32)
    need = std::max(need, fw_exec_workspace(n, o.bs ? o.bs : default_bs_for(n, APSP_DTYPE_U16X2),
                                            APSP_DTYPE_U16X2, D, P));
  return need;
}

}  // namespace apsp

extern "C" size_t apsp_fw_workspace_size(int n, const apsp_options* opt) {
  return fw_workspace_need(n, opt, nullptr, nullptr);  // null pointers count as aligned
}

extern "C" size_t apsp_fw_workspace_size_for(int n, const apsp_options* opt, const float* D, const int32_t* P) {
  return fw_workspace_need(n, opt, D, P);
}

namespace apsp {

// Scan W and decide the arithmetic. Synchronises `s` once.
static apsp_status scan_and_choose(const float* W, int n, int want, WeightStats* dstats, cudaStream_t s, int* dtype_out,
                                   int* graph_int) {
  if (cudaMemsetAsync(dstats, 0, sizeof(WeightStats), s) != cudaSuccess) return APSP_ECUDA;
  scan_weights_kernel<<<elementwise_grid((size_t)n * n), 256, 0, s>>>(W, n, dstats);
  WeightStats hs;
  if (cudaMemcpyAsync(&hs, dstats, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess) return APSP_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return APSP_ECUDA;
  if (hs.n_negative || hs.n_nan) return APSP_EINVAL;
  float mx;
  std::memcpy(&mx, &hs.max_bits, sizeof(mx));
  const bool eligible = u16_eligible(hs.n_fraction == 0, hs.n_inf == 0, mx, n);
  if (want == APSP_DTYPE_U16X2 && !eligible) return APSP_EINVAL;
  *graph_int = hs.n_fraction == 0;
  *dtype_out = (want == APSP_DTYPE_F32) ? APSP_DTYPE_F32 : (eligible ? APSP_DTYPE_U16X2 : APSP_DTYPE_F32);
  return APSP_OK;
}

// Run the block rounds with the arithmetic already chosen (no input scan).
apsp_status fw_exec(const float* W, float* D, int32_t* P, int n, int bs, int dtype, int graph_int, int flags,
                    void* workspace, size_t workspace_bytes, apsp_run_info* info, cudaStream_t s) {
  bool p_in_place = false;
  const Plan pl = plan_for(n, bs, dtype, D, P, &p_in_place);
  void* ws = workspace;
  bool own_ws = false;
  if (ws == nullptr) {
    if (cudaMallocAsync(&ws, std::max<size_t>(pl.ws_total, 256), s) != cudaSuccess) {
      cudaGetLastError();
      return APSP_ENOMEM;
    }
    own_ws = true;
  } else if (workspace_bytes < pl.ws_total) {
    return APSP_ENOMEM;
  }

  char* wsb = static_cast<char*>(ws);
  int32_t* Pw = p_in_place ? P : reinterpret_cast<int32_t*>(wsb + pl.ws_p);
  const size_t quads = (size_t)pl.n_pad * (pl.n_pad / 4);
  RoundMax* rmax = reinterpret_cast<RoundMax*>(wsb + kRoundMaxOffset);
  PhaseTimer tm;
  tm.s = s;
  tm.on = (flags & APSP_FLAG_TIME_PHASES) != 0;
  int aux = 0;
  cudaError_t e = cudaSuccess;
  if (dtype == APSP_DTYPE_F32) {
    float* Dw = pl.in_place ? D : reinterpret_cast<float*>(wsb + pl.ws_d);
    init_f32_kernel<<<elementwise_grid(quads), 256, 0, s>>>(W, n, Dw, Pw, pl.n_pad, &rmax->fault);
    ++aux;
    e = launch_rounds<F32T>(Dw, Pw, pl.n_pad, pl.bs, s, tm, rmax,
                            graph_int, reinterpret_cast<float*>(wsb + pl.ws_pan), wsb + pl.ws_diag, flags);
    if (e == cudaSuccess && !pl.in_place) {
      copy_out_kernel<float><<<elementwise_grid((size_t)n * n), 256, 0, s>>>(Dw, pl.n_pad, D, n);
      ++aux;
    }
  } else {
    uint16_t* Dw = reinterpret_cast<uint16_t*>(wsb + pl.ws_d);
    init_u16_kernel<<<elementwise_grid(quads), 256, 0, s>>>(W, n, Dw, Pw, pl.n_pad, &rmax->fault);
    ++aux;
    e = launch_rounds<U16T>(Dw, Pw, pl.n_pad, pl.bs, s, tm, rmax, 0,
                            reinterpret_cast<float*>(wsb + pl.ws_pan), wsb + pl.ws_diag, flags);
    if (e == cudaSuccess) {
      widen_u16_kernel<<<elementwise_grid((size_t)n * n), 256, 0, s>>>(Dw, pl.n_pad, D, n);
      ++aux;
    }
  }
  if (e == cudaSuccess && !p_in_place) {
    copy_out_kernel<int32_t><<<elementwise_grid((size_t)n * n), 256, 0, s>>>(Pw, pl.n_pad, P, n);
    ++aux;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  float ms[3];
  tm.finish(ms);
  if (own_ws) cudaFreeAsync(ws, s);
  if (e != cudaSuccess) return APSP_ECUDA;
  if (info) {
    info->bs_used = pl.bs;
    info->dtype_used = dtype;
    info->rounds = pl.n_pad / pl.bs;
    info->n_pad = pl.n_pad;
    info->launches += aux + tm.other + tm.launches[0] + tm.launches[1] + tm.launches[2];
    for (int q = 0; q < 3; ++q) {
      info->phase_launches[q] = tm.launches[q];
      info->phase_ms[q] = ms[q];
    }
  }
  return APSP_OK;
}

apsp_status fw_run(const float* W, float* D, int32_t* P, int n, const apsp_options* opt, void* workspace,
                   size_t workspace_bytes, apsp_run_info* info, cudaStream_t s) {
  apsp_options o = opt ? *opt : default_options();
  if (n < 1 || !W || !D || !P) return APSP_EINVAL;
  if (o.bs != 0 && !valid_bs(o.bs)) return APSP_EINVAL;
  if (o.dtype < APSP_DTYPE_AUTO || o.dtype > APSP_DTYPE_U16X2) return APSP_EINVAL;
  if (!o.validate && o.dtype != APSP_DTYPE_F32) return APSP_EINVAL;
  if (n > 65536) return APSP_EINVAL;
  if (workspace && ((uintptr_t)workspace & 255) != 0) return APSP_EINVAL;
  // A caller workspace must hold what either possible arithmetic needs for these D and P;
  // checked before anything is enqueued.
  if (workspace && workspace_bytes < fw_workspace_need(n, &o, D, P)) return APSP_ENOMEM;
  if (info) std::memset(info, 0, sizeof(*info));

  // Scan counters: the caller's workspace head, or a small stream-ordered buffer.
  int dtype = APSP_DTYPE_F32;
  int graph_int = 0;  // unknown without the scan: phase 3 then takes the generic P search
  if (o.validate) {
    void* sbuf = workspace;
    if (sbuf == nullptr) {
      if (cudaMallocAsync(&sbuf, 256, s) != cudaSuccess) {
        cudaGetLastError();
        return APSP_ENOMEM;
      }
    } else if (workspace_bytes < sizeof(WeightStats)) {
      return APSP_ENOMEM;
    }
    apsp_status st = scan_and_choose(W, n, o.dtype, reinterpret_cast<WeightStats*>(sbuf), s, &dtype, &graph_int);
    if (workspace == nullptr) cudaFreeAsync(sbuf, s);
    if (st != APSP_OK) return st;
    if (info) info->launches = 1;
  }
  if (o.bs == 0) o.bs = default_bs_for(n, dtype);
  return fw_exec(W, D, P, n, o.bs, dtype, graph_int, o.flags, workspace, workspace_bytes, info, s);
}

}  // namespace apsp

extern "C" apsp_status apsp_fw_ex(const float* W, float* D, int32_t* P, int n, const apsp_options* opt, void* workspace,
                                  size_t workspace_bytes, apsp_run_info* info, void* stream) {
  return fw_run(W, D, P, n, opt, workspace, workspace_bytes, info, static_cast<cudaStream_t>(stream));
}

extern "C" apsp_status apsp_fw(const float* W, float* D, int32_t* P, int n, void* stream) {
  return fw_run(W, D, P, n, nullptr, nullptr, 0, nullptr, static_cast<cudaStream_t>(stream));
}

extern "C" apsp_status apsp_device_status(int clear) {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_apsp_fault, sizeof(v)) != cudaSuccess) return APSP_ECUDA;
  if (clear && v) {
    const unsigned zero = 0;
    if (cudaMemcpyToSymbol(g_apsp_fault, &zero, sizeof(zero)) != cudaSuccess) return APSP_ECUDA;
  }
  return (v & kFaultPanelCopyTimeout) ? APSP_ETIMEOUT : APSP_OK;
}

namespace apsp {

// Streams that carry apsp_fw_host's copies in row chunks, so that several copy
// engines move one matrix at once (created once per device, never destroyed).
constexpr int kCopyStreams = 4;
static cudaError_t copy_streams(cudaStream_t** out) {
  static std::once_flag once[kMaxDevices];
  static cudaStream_t streams[kMaxDevices][kCopyStreams];
  static cudaError_t errs[kMaxDevices];
  const int dev = current_device();
  if (dev < 0) return cudaErrorInvalidDevice;
  std::call_once(once[dev], [dev] {
    errs[dev] = cudaSuccess;
    for (int c = 0; c < kCopyStreams && errs[dev] == cudaSuccess; ++c)
      errs[dev] = cudaStreamCreateWithFlags(&streams[dev][c], cudaStreamNonBlocking);
  });
  *out = streams[dev];
  return errs[dev];
}

// Copy `rows` rows of `row_bytes` bytes in kCopyStreams row chunks, each on its
// own stream, ordered after everything enqueued on `s` so far; `s` then waits
// for all chunks. ev: kCopyStreams + 1 events.
static cudaError_t chunked_copy(void* dst, const void* src, size_t rows, size_t row_bytes, cudaMemcpyKind kind,
                                cudaStream_t s, cudaStream_t* cs, cudaEvent_t* ev) {
  cudaError_t e = cudaEventRecord(ev[kCopyStreams], s);
  const size_t per = (rows + kCopyStreams - 1) / kCopyStreams;
  for (int c = 0; c < kCopyStreams && e == cudaSuccess; ++c) {
    const size_t r0 = std::min(rows, (size_t)c * per), r1 = std::min(rows, r0 + per);
    e = cudaStreamWaitEvent(cs[c], ev[kCopyStreams], 0);
    if (e == cudaSuccess && r1 > r0)
      e = cudaMemcpyAsync(static_cast<char*>(dst) + r0 * row_bytes, static_cast<const char*>(src) + r0 * row_bytes,
                          (r1 - r0) * row_bytes, kind, cs[c]);
    if (e == cudaSuccess) e = cudaEventRecord(ev[c], cs[c]);
  }
  for (int c = 0; c < kCopyStreams && e == cudaSuccess; ++c) e = cudaStreamWaitEvent(s, ev[c], 0);
  return e;
}

}  // namespace apsp

extern "C" apsp_status apsp_fw_host(const float* W, float* D, int32_t* P, int n, const apsp_options* opt,
                                    apsp_run_info* info, void* stream) {
  if (n < 1 || !W || !D || !P) return APSP_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)n * n * sizeof(float);
  cudaStream_t* cs = nullptr;
  if (copy_streams(&cs) != cudaSuccess) return APSP_ECUDA;
  cudaEvent_t ev[kCopyStreams + 1] = {};
  for (auto& e : ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      for (auto& x : ev)
        if (x) cudaEventDestroy(x);
      return APSP_ECUDA;
    }
  // W goes straight into the device D and the solve runs in place (W may alias D).
  float* dD = nullptr;
  int32_t* dP = nullptr;
  apsp_status st = APSP_OK;
  if (cudaMallocAsync(&dD, bytes, s) != cudaSuccess || cudaMallocAsync(&dP, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    st = APSP_ENOMEM;
  }
  const size_t row = (size_t)n * sizeof(float);
  if (st == APSP_OK && chunked_copy(dD, W, n, row, cudaMemcpyHostToDevice, s, cs, ev) != cudaSuccess) st = APSP_ECUDA;
  if (st == APSP_OK) st = fw_run(dD, dD, dP, n, opt, nullptr, 0, info, s);
  if (st == APSP_OK) {
    if (chunked_copy(D, dD, n, row, cudaMemcpyDeviceToHost, s, cs, ev) != cudaSuccess ||
        chunked_copy(P, dP, n, row, cudaMemcpyDeviceToHost, s, cs, ev) != cudaSuccess)
      st = APSP_ECUDA;
  }
  if (dD) cudaFreeAsync(dD, s);
  if (dP) cudaFreeAsync(dP, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && st == APSP_OK) st = APSP_ECUDA;
  for (auto& e : ev) cudaEventDestroy(e);
  if (st == APSP_ENOMEM) return st;
  if (st == APSP_OK) st = apsp_device_status(1);
  return st;
}
