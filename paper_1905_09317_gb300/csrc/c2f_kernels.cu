// c2f_kernels.cu -- the GB300 kernels of the fire-growth path.
//
//   k_cell_prep / k_hour_prep   hoisted per-cell and per-hour FBP terms
//   k_ros_table   (K1)  per (cell, hour): FBP HROS/BROS/LB, Eqs. (1)-(4), the 8
//                       axis rates as 2^32 fixed-point per-period increments
//   k_ignite      (K2)  Step 1 of Alg. 1: ignition cell per replica
//   k_frontier    (K3)  Step 2 of Alg. 1 for whole replicas: send / receive /
//                       burn-out per fire period, one CTA per replica
//   k_burn_prob   (K4)  burn-probability counts over replicas
//   k_compare_hours / k_compare_final   scar comparison metrics of Sec. 4.1
// plus landscape set-up (burnable bit plane and list) and result export.
//
// Frontier semantics (Sec. 3.1, 3.4, A5; Alg. 1):
//   - a cell ignited in period t advances each open axis from period t+1 by
//     its per-period increment while the neighbour on that axis is Available
//     at the start of the period; when the progress reaches the axis length
//     (the centre-to-centre distance) a message is sent and the axis closes;
//   - a messaged Available cell ignites in that period if HROS * f exceeds
//     the threshold (f: the perturbation of the receiver for the hour);
//   - at the end of a period a burning cell with no Available neighbour, or
//     (delta > 0) with HROS * f < delta, becomes Burned;
//   - the work count adds the number of burning cells at the start of each
//     period.
// The increment of an axis is constant within a weather hour, so within an
// hour the period at which an axis reaches its neighbour's centre is an
// integer function of the progress at the start of the hour; the kernel
// stores that crossing period (as an offset in the hour) instead of adding
// the increment every period, and only visits periods at which something
// happens.  All progress arithmetic is int64, so the crossing periods are the
// ones the period-by-period loop produces.
#include <cstdint>
#include <mutex>
#include <type_traits>

#include "c2f_fbp.cuh"

namespace c2f {

// host: fill the per-device constant tables (math coefficients, fuel table)
cudaError_t upload_constants() {
  MathConstants mc;
  make_math_constants(&mc);
  FuelCoef ft[F_NCODES];
  make_fuel_table(ft);
  cudaError_t e = cudaMemcpyToSymbol(g_mc, &mc, sizeof mc);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_fuel, ft, sizeof ft);
  if (e == cudaSuccess) {
    k_math_tables<<<1, 256>>>();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e;
}

// once per device and process, for every entry point that launches kernels
cudaError_t init_device_constants(int device) {
  static std::once_flag once[64];
  static cudaError_t err[64];
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::call_once(once[device], [device] { err[device] = upload_constants(); });
  return err[device];
}

// axis k = 0..7 at 45 k degrees counter-clockwise from east: (row, col) offsets
// E (0,+1), NE (-1,+1), N (-1,0), NW (-1,-1), W (0,-1), SW (+1,-1), S (+1,0), SE (+1,+1),
// kept as offset + 1 in the nibbles of one immediate: lanes index them with
// different k, which a __constant__ table would serve one address at a time
__device__ __forceinline__ int axis_dr(int k) { return (int)((0x22210001u >> (4 * k)) & 0xFu) - 1; }
__device__ __forceinline__ int axis_dc(int k) { return (int)((0x21000122u >> (4 * k)) & 0xFu) - 1; }

// bit 0 of each byte of x, gathered into bits 0..3 (byte 0 -> bit 0)
__device__ __forceinline__ uint32_t byte_lsbs(uint32_t x) {
  return (((x & 0x01010101u) * 0x00204081u) >> 21) & 0xFu;
}

// ------------------------------------------------------------------ set-up
// burnable plane (bit per cell, rows padded to 32-bit words) and per-word counts
__global__ void k_burnable_plane(const uint8_t *__restrict__ fuel, const uint8_t *__restrict__ unb,
                                 int32_t rows, int32_t cols, int32_t wpr, uint32_t *plane,
                                 int32_t *word_count) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= (int64_t)rows * wpr) return;
  const int32_t row = (int32_t)(w / wpr), cw = (int32_t)(w % wpr);
  uint32_t bits = 0;
  for (int b = 0; b < 32; ++b) {
    const int32_t col = cw * 32 + b;
    if (col >= cols) break;
    const int64_t cell = (int64_t)row * cols + col;
    const bool ok = fuel[cell] != 0 && !(unb && unb[cell]);
    bits |= (ok ? 1u : 0u) << b;
  }
  plane[w] = bits;
  word_count[w] = __popc(bits);
}

// exclusive scan of the per-word counts, one block (set-up only)
__global__ void k_scan_counts(const int32_t *__restrict__ cnt, int64_t n, int32_t *offs,
                              int32_t *total) {
  __shared__ int32_t s_part[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int64_t per = (n + T - 1) / T;
  const int64_t b = per * t, e = (b + per < n) ? b + per : n;
  int32_t acc = 0;
  for (int64_t i = b; i < e; ++i) acc += cnt[i];
  s_part[t] = acc;
  __syncthreads();
  if (t == 0) {
    int32_t run = 0;
    for (int i = 0; i < T; ++i) { const int32_t v = s_part[i]; s_part[i] = run; run += v; }
    *total = run;
  }
  __syncthreads();
  int32_t run = s_part[t];
  for (int64_t i = b; i < e; ++i) { offs[i] = run; run += cnt[i]; }
}

__global__ void k_burnable_list(const uint32_t *__restrict__ plane, const int32_t *__restrict__ offs,
                                int32_t rows, int32_t cols, int32_t wpr, int32_t *list) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= (int64_t)rows * wpr) return;
  const int32_t row = (int32_t)(w / wpr), cw = (int32_t)(w % wpr);
  uint32_t bits = plane[w];
  int32_t o = offs[w];
  while (bits) {
    const int b = __ffs(bits) - 1;
    bits &= bits - 1;
    list[o++] = row * cols + cw * 32 + b;
  }
}

// ------------------------------------------------------------------ K1 prep
__global__ void k_cell_prep(const float *__restrict__ slope, const float *__restrict__ aspect,
                            int64_t n, CellPrep *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  CellPrep cp;
  cell_prep(slope ? (double)slope[i] : 0.0, aspect ? (double)aspect[i] : 0.0, &cp);
  out[i] = cp;
}

// one thread per hour: weather-only terms
__global__ void k_hour_prep(const double *__restrict__ weather, int32_t hours, double o1_curing,
                            HourPrep *out) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= hours) return;
  const double *w = weather + (size_t)h * 4;
  const double cf = curing_factor(o1_curing);
  hour_prep(w[0], w[1], w[2], w[3], cf, &out[h]);
}

// ------------------------------------------------------------------ K1

// Cells grouped by (fuel code, slope > 0) so that the lanes of a warp take the
// same branches of the FBP code (set-up, once per landscape): a per-bucket
// count, an exclusive scan, then a scatter; the order inside a bucket is
// immaterial because every cell writes its own table row.
__device__ __forceinline__ int order_bucket(const uint8_t *fuel, const float *slope,
                                            const uint32_t *burnable, int32_t cols, int32_t wpr,
                                            int64_t cell) {
  const int32_t row = (int32_t)(cell / cols), col = (int32_t)(cell % cols);
  const bool burn = (burnable[(int64_t)row * wpr + (col >> 5)] >> (col & 31)) & 1u;
  if (!burn) return 0;
  const bool sloped = slope && slope[cell] > 0.0f;
  return 2 * (int)fuel[cell] + (sloped ? 1 : 0);
}

__global__ void k_order_count(const uint8_t *fuel, const float *slope, const uint32_t *burnable,
                              int32_t rows, int32_t cols, int32_t wpr, int32_t *counts) {
  __shared__ int32_t h[kOrderBuckets];
  if (threadIdx.x < kOrderBuckets) h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell < (int64_t)rows * cols)
    atomicAdd(&h[order_bucket(fuel, slope, burnable, cols, wpr, cell)], 1);
  __syncthreads();
  if (threadIdx.x < kOrderBuckets && h[threadIdx.x]) atomicAdd(&counts[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_order_scan(int32_t *counts_to_cursor) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int32_t run = 0;
    for (int b = 0; b < kOrderBuckets; ++b) {
      const int32_t c = counts_to_cursor[b];
      counts_to_cursor[b] = run;
      run += c;
    }
  }
}

__global__ void k_order_scatter(const uint8_t *fuel, const float *slope, const uint32_t *burnable,
                                int32_t rows, int32_t cols, int32_t wpr, int32_t *cursor,
                                int32_t *order) {
  __shared__ int32_t h[kOrderBuckets], base[kOrderBuckets];
  if (threadIdx.x < kOrderBuckets) h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int b = -1, local = 0;
  if (cell < (int64_t)rows * cols) {
    b = order_bucket(fuel, slope, burnable, cols, wpr, cell);
    local = atomicAdd(&h[b], 1);
  }
  __syncthreads();
  if (threadIdx.x < kOrderBuckets && h[threadIdx.x]) base[threadIdx.x] = atomicAdd(&cursor[threadIdx.x], h[threadIdx.x]);
  __syncthreads();
  if (b >= 0) order[base[b] + local] = (int32_t)cell;
}

// the 8 axis rates and HROS of one burnable cell at one hour
// (const_ros > 0: the deterministic test rates -- all 8 axes at const_ros, or,
// with const_bros > 0 or const_lb > 1, the ellipse of HROS = const_ros,
// BROS = const_bros (0: const_ros), LB = const_lb headed along the hour's wind)
__device__ __forceinline__ double row_rates(int fuel, const float *slope, int64_t cell,
                                            const CellPrep &cp, const HourPrep &hp, double pcf,
                                            double const_ros, double const_bros, double const_lb,
                                            int ellipse_mode, double ros[8]) {
  if (pos(const_ros)) {
    if (pos(const_bros) || gt_c(const_lb, 1.0)) {
      FbpOut o;
      ellipse_axes(const_ros, pos(const_bros) ? const_bros : const_ros, gt_c(const_lb, 1.0) ? const_lb : 1.0,
                   hp.sin_w, hp.cos_w, ellipse_mode, &o);
#pragma unroll
      for (int k = 0; k < 8; ++k) ros[k] = o.ros[k];
      return const_ros;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) ros[k] = const_ros;
    return const_ros;
  }
  const double gs = slope ? (double)slope[cell] : 0.0;
  FbpOut o;
  fbp_row(fuel, gs, cp, hp, pcf, ellipse_mode, &o);
#pragma unroll
  for (int k = 0; k < 8; ++k) ros[k] = o.ros[k];
  return o.hros;
}

// a table row: the 8 per-period increments B_k = fixed(ros_k * dt * 2^32) in one
// 64-byte line (four 16-byte stores), HROS beside it in its own array
__device__ __forceinline__ void row_store(int64_t *row, double *hros_at, const double ros[8],
                                          double hr, double dt2p32) {
  longlong2 *dst = reinterpret_cast<longlong2 *>(row);
#pragma unroll
  for (int k = 0; k < 8; k += 2)
    dst[k / 2] = make_longlong2(fixed_of(__dmul_rn(ros[k], dt2p32)), fixed_of(__dmul_rn(ros[k + 1], dt2p32)));
  *hros_at = hr;
}

// nanoseconds of the GPU's global timer
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// one launch-trace record (c2f_trace); records past the capacity are counted, not written
__device__ __forceinline__ void trace_record(const TraceArgs &tr, uint32_t kind, uint32_t aux, long long tag,
                                             unsigned long long t0, unsigned long long t1) {
  const unsigned long long i = atomicAdd(tr.cursor, 1ull);
  if (i < (unsigned long long)tr.cap) {
    uint32_t smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    unsigned long long *p = tr.rec + 4 * i;
    p[0] = (unsigned long long)kind | ((unsigned long long)smid << 8) | ((unsigned long long)aux << 32);
    p[1] = (unsigned long long)tag;
    p[2] = t0;
    p[3] = t1;
  }
}

__global__ void __launch_bounds__(128) k_ros_table(RosTableArgs a) {
  const int64_t n = (int64_t)a.rows * a.cols;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool traced = a.trace.rec != nullptr && threadIdx.x == 0;   // thread 0 stands for its CTA
  const unsigned long long t_start = traced ? global_ns() : 0ull;
  if (t >= n) return;
  const int64_t cell = a.order ? (int64_t)a.order[t] : t;
  const int h = a.hour0 + blockIdx.y;
  const int32_t row = (int32_t)(cell / a.cols), col = (int32_t)(cell % a.cols);
  const bool burn = (a.burnable[(int64_t)row * a.wpr + (col >> 5)] >> (col & 31)) & 1u;
  double ros[8];
  double hr = 0.0;
  if (!burn) {
#pragma unroll
    for (int k = 0; k < 8; ++k) ros[k] = 0.0;
  } else {
    hr = row_rates(a.fuel[cell], a.slope, cell, a.cell[cell], a.hour[h], a.pcf, a.const_ros,
                   a.const_bros, a.const_lb, a.ellipse_mode, ros);
  }
  const size_t idx = (size_t)h * n + cell;
  if (a.base) {
    double scratch;
    row_store(a.base + idx * 8, a.hros ? a.hros + idx : &scratch, ros, hr, a.dt2p32);
  } else if (a.hros) {
    a.hros[idx] = hr;
  }
  if (a.ros8) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a.ros8[(size_t)cell * 8 + k] = ros[k];
  }
  if (traced) trace_record(a.trace, kTraceTable, (uint32_t)h, a.trace.tag, t_start, global_ns());
}

// ------------------------------------------------------------------ K2
__global__ void k_ignite(const SimJob *jobs, int32_t job) {
  const SimJob &J = jobs[job];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= J.n_replicas) return;
  int32_t ic = J.ignition_cell;
  if (J.ignition_mode == 1) {
    const U4 x = philox4x32_10(U4{(uint32_t)r, 0u, 0u, 1u}, (uint32_t)J.seed,
                               (uint32_t)(J.seed >> 32));
    const uint64_t idx = ((uint64_t)x.x * (uint64_t)(uint32_t)J.n_burnable) >> 32;
    ic = J.burnable_list[idx];
  }
  J.ign_cell[r] = ic;
  if (J.n_scen > 1) {   // Sec. 3.1 (3): the first s with x0 < T_s, x0 from counter (r, 0, 0, 2)
    const U4 x = philox4x32_10(U4{(uint32_t)r, 0u, 0u, 2u}, (uint32_t)J.seed,
                               (uint32_t)(J.seed >> 32));
    int32_t s = 0;
    while (s < J.n_scen - 1 && (uint64_t)x.x >= J.scen_thr[s]) ++s;
    J.scen[r] = s;
  }
}

// ------------------------------------------------------------------ K3
__device__ __forceinline__ bool plane_bit(const uint32_t *p, int32_t wpr, int32_t r, int32_t c) {
  return (p[r * wpr + (c >> 5)] >> (c & 31)) & 1u;
}

__device__ __forceinline__ uint32_t min_byte8(uint64_t v) {
  uint32_t m = __vminu4((uint32_t)v, (uint32_t)(v >> 32));
  m = __vminu4(m, m >> 16);
  m = __vminu4(m, m >> 8);
  return m & 0xFFu;
}

__device__ __forceinline__ int64_t axis_len(const SimJob &J, int k) {
  return (k & 1) ? J.d_diag : J.d_orth;
}

// smallest n >= 1 with n * inc >= rem, for callers that know 64 * inc >= rem
// (a crossing within the hour: at most 60 periods).  Six halving steps of
// exact int64 products; a conversion of int64 operands to floating point costs
// several times more on this GPU.
__device__ __forceinline__ int32_t ceil_div_small(int64_t rem, int64_t inc) {
  int32_t n = 0;   // n * inc < rem, or n = 0
#pragma unroll
  for (int b = 5; b >= 0; --b) {
    const int32_t t = n + (1 << b);
    if ((int64_t)t * inc < rem) n = t;
  }
  return n + 1;
}

// The frontier's two binary64 tests are kept out of line: inlined, the
// compiler issues their FP64 instructions (predicated off) in every round and
// set-up pass even when no threshold or delta is set, and each of them waits
// for the FP64 pipe, which a table build running beside the frontier keeps
// busy.  Called only when a threshold (receive) or a delta (burn-out) is set.

// receive test of a messaged Available cell (Sec. 3.1): HROS * f > threshold
__device__ __noinline__ bool receive_ok(const SimJob &J, int32_t r, int64_t j, int32_t h, int64_t n) {
  if (J.thr < 0.0) return true;
  const double hr = __ldcg(J.hros + (size_t)h * n + j);
  if (J.thr == 0.0) {
    if (hr > 1e-200) return true;   // f >= exp(-5.9) for sigma <= 1, so HROS * f > 0
    if (!(hr > 0.0)) return false;
  }
  const float f = noise_factor(J.seed, (uint32_t)r, (uint32_t)j, (uint32_t)h, J.sigma);
  return __dmul_rn(hr, (double)f) > J.thr;
}

// A5 (i): the cell's HROS * f this hour is below delta
__device__ __noinline__ bool below_delta(const double *hrosh, int64_t cell, float f, double delta) {
  return __dmul_rn(__ldcg(hrosh + cell), (double)f) < delta;
}

__device__ __forceinline__ int64_t find_job(const int64_t *begin, int32_t n, int64_t item) {
  int32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (begin[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint32_t warp_min(uint32_t v) {
  return __reduce_min_sync(0xffffffffu, v);   // one warp-wide reduction instruction
}

// min over the 8 lanes of this lane's group
__device__ __forceinline__ uint32_t group_min(uint32_t v) {
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// a per-lane flag over the 8 lanes of this lane's group, as an 8-bit mask (bit k = lane k)
__device__ __forceinline__ uint32_t group_bits(bool b) {
  const uint32_t bal = __ballot_sync(0xffffffffu, b);
  return (bal >> (threadIdx.x & 24)) & 0xFFu;
}

__device__ __forceinline__ uint32_t rc_pack(int32_t r, int32_t c) {
  return ((uint32_t)r << 16) | (uint32_t)c;
}

// a table row into L2 ahead of its use
__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// a 64-byte table row into this SM's L1 ahead of its use (both 32-byte
// sectors); only for tables that no warp writes while the frontier runs
__device__ __forceinline__ void prefetch_row_l1(const int64_t *row) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(row));
  asm volatile("prefetch.global.L1 [%0];" ::"l"(row + 4));
}

// chunk state, read at device scope from L2.  A relaxed load suffices: a warp
// reads a chunk's rows (with L2 loads, __ldcg) only after a branch on the
// state it loaded has resolved, and the computing warp made its rows visible
// device-wide (__threadfence) before it set the state.  An acquire load would
// also invalidate the SM's L1 on every check.
__device__ __forceinline__ uint32_t ld_state(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// waits for a table chunk that another warp is computing give up after
// FrontierArgs::wait_limit polls (this many when it is 0: about a second);
// the replica then stops with status 4 (a bounded wait ran out)
constexpr uint32_t kChunkSpinLimit = 1u << 23;

// On-demand table rows: the rows at hour h of the 32 cells of bit-plane word w
// (one lane per cell, all 32 lanes of the warp), then the chunk's state goes
// to done once every lane's stores are visible device-wide.
__device__ __forceinline__ void table_chunk(const SimJob &J, int32_t h, int32_t w) {
  const int lane = threadIdx.x & 31;
  const int32_t row = w / J.wpr, cw = w - row * J.wpr;
  const int32_t col = cw * 32 + lane;
  if (col < J.cols && ((__ldg(&J.burnable[w]) >> lane) & 1u)) {
    const int64_t n = (int64_t)J.rows * J.cols;
    const int64_t cell = (int64_t)row * J.cols + col;
    double ros[8];
    const double hr = row_rates(__ldg(&J.fuel[cell]), J.slope, cell, J.cell[cell], J.hour[h], J.pcf,
                                J.const_ros, J.const_bros, J.const_lb, J.ellipse_mode, ros);
    const size_t idx = (size_t)h * n + cell;
    row_store(J.base + idx * 8, J.hros + idx, ros, hr, J.dt2p32);
  }
  __threadfence();
  __syncwarp();
  if (lane == 0) atomicExch(J.chunk_state + (size_t)h * J.rows * J.wpr + w, 2u);
  __syncwarp();
}

// 32-bit atomics on words known to lie in shared memory
__device__ __forceinline__ uint32_t atom_and_shared(uint32_t *p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.shared.and.b32 %0, [%1], %2;"
               : "=r"(old) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ uint32_t atom_or_shared(uint32_t *p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.shared.or.b32 %0, [%1], %2;"
               : "=r"(old) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ int32_t atom_exch_shared(int32_t *p, int32_t v) {
  int32_t old;
  asm volatile("atom.shared.exch.b32 %0, [%1], %2;"
               : "=r"(old) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(v) : "memory");
  return old;
}

// The replica's Available and Burned bit planes.  With WIN, a window of
// kWinRows x (32 kWinWords) cells around the ignition cell lives in shared
// memory and the rest of the grid in global memory; without it, all in global
// memory.  Accessors hand out a pointer to the 32-bit word holding (r, c).
template <bool WIN>
struct Planes {
  uint32_t *sav, *sbr;   // shared-memory windows
  uint32_t *gav, *gbr;   // full planes, global memory
  int32_t r0, w0, wpr;
  __device__ __forceinline__ bool in_win(int32_t r, int32_t w) const {
    if constexpr (WIN) return (uint32_t)(r - r0) < (uint32_t)kWinRows && (uint32_t)(w - w0) < (uint32_t)kWinWords;
    else return false;
  }
  __device__ __forceinline__ uint32_t *avw(int32_t r, int32_t c) const {
    const int32_t w = c >> 5;
    if (in_win(r, w)) return sav + (r - r0) * kWinWords + (w - w0);
    return gav + r * wpr + w;
  }
  __device__ __forceinline__ uint32_t *brw(int32_t r, int32_t c) const {
    const int32_t w = c >> 5;
    if (in_win(r, w)) return sbr + (r - r0) * kWinWords + (w - w0);
    return gbr + r * wpr + w;
  }
  __device__ __forceinline__ bool avail(int32_t r, int32_t c) const { return (*avw(r, c) >> (c & 31)) & 1u; }
  __device__ __forceinline__ bool burned(int32_t r, int32_t c) const { return (*brw(r, c) >> (c & 31)) & 1u; }
  // ignition: clears the Available bit; true for the one caller that cleared it
  // (a word of the window is changed with a shared-memory atomic, the others
  // in global memory: an atomic on a generic address costs more than either)
  __device__ __forceinline__ bool take(int32_t r, int32_t c) const {
    const uint32_t bit = 1u << (c & 31);
    const int32_t w = c >> 5;
    if (in_win(r, w)) return (atom_and_shared(sav + (r - r0) * kWinWords + (w - w0), ~bit) & bit) != 0;
    return (atomicAnd(gav + r * wpr + w, ~bit) & bit) != 0;
  }
  // burn-out: sets the Burned bit; true for the one caller that set it
  __device__ __forceinline__ bool burn(int32_t r, int32_t c) const {
    const uint32_t bit = 1u << (c & 31);
    const int32_t w = c >> 5;
    if (in_win(r, w)) return (atom_or_shared(sbr + (r - r0) * kWinWords + (w - w0), bit) & bit) == 0;
    return (atomicOr(gbr + r * wpr + w, bit) & bit) == 0;
  }
  // the Available neighbours of (r, c) as an 8-bit mask, bit k = axis k
  // (neighbours outside the grid are not Available)
  __device__ __forceinline__ uint32_t avail_mask(int32_t rows, int32_t cols, int32_t r, int32_t c) const {
    if constexpr (WIN) {
      // the common case, as in any_avail_nbr: three window rows, funnel shifts
      const int32_t il = ((c - 1) >> 5) - w0, ih = ((c + 1) >> 5) - w0;
      if (c >= 1 && r >= 1 && r + 1 < rows && (uint32_t)(r - 1 - r0) < (uint32_t)(kWinRows - 2) &&
          (uint32_t)il < (uint32_t)kWinWords && (uint32_t)ih < (uint32_t)kWinWords) {
        const uint32_t *p = sav + (r - 1 - r0) * kWinWords;
        const uint32_t sh = (uint32_t)(c - 1) & 31u;
        const uint32_t up = __funnelshift_r(p[il], p[ih], sh) & 7u;                  // NW N NE
        const uint32_t mid = __funnelshift_r(p[kWinWords + il], p[kWinWords + ih], sh) & 7u;   // W . E
        const uint32_t dn = __funnelshift_r(p[2 * kWinWords + il], p[2 * kWinWords + ih], sh) & 7u;  // SW S SE
        return ((mid >> 2) & 1u) | (((up >> 2) & 1u) << 1) | (((up >> 1) & 1u) << 2) | ((up & 1u) << 3) |
               ((mid & 1u) << 4) | ((dn & 1u) << 5) | (((dn >> 1) & 1u) << 6) | (((dn >> 2) & 1u) << 7);
      }
    }
    uint32_t m = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int32_t nr = r + axis_dr(q), nc = c + axis_dc(q);
      if (nr >= 0 && nr < rows && nc >= 0 && nc < cols && avail(nr, nc)) m |= 1u << q;
    }
    return m;
  }
  // some neighbour of (r, c) is still Available
  __device__ __forceinline__ bool any_avail_nbr(int32_t rows, int32_t cols, int32_t r, int32_t c) const {
    if constexpr (WIN) {
      // the common case: the 3 x 3 block lies inside the grid and the window;
      // a row's three bits come out of two adjacent window words by one funnel
      // shift (bits past the last column are 0 in the plane)
      const int32_t il = ((c - 1) >> 5) - w0, ih = ((c + 1) >> 5) - w0;
      if (c >= 1 && r >= 1 && r + 1 < rows && (uint32_t)(r - 1 - r0) < (uint32_t)(kWinRows - 2) &&
          (uint32_t)il < (uint32_t)kWinWords && (uint32_t)ih < (uint32_t)kWinWords) {
        const uint32_t *p = sav + (r - 1 - r0) * kWinWords;
        const uint32_t sh = (uint32_t)(c - 1) & 31u;
        const uint32_t up = __funnelshift_r(p[il], p[ih], sh) & 7u;
        const uint32_t mid = __funnelshift_r(p[kWinWords + il], p[kWinWords + ih], sh) & 5u;
        const uint32_t dn = __funnelshift_r(p[2 * kWinWords + il], p[2 * kWinWords + ih], sh) & 7u;
        return (up | mid | dn) != 0u;
      }
    }
    uint32_t words[3][2];
    const int32_t c0 = c > 0 ? c - 1 : 0, c1 = c + 1 < cols ? c + 1 : cols - 1;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int32_t rr = r - 1 + d;
      const bool ok = rr >= 0 && rr < rows;
      words[d][0] = ok ? *avw(rr, c0) : 0u;
      words[d][1] = ok ? *avw(rr, c1) : 0u;
    }
    bool any = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int dc = -1; dc <= 1; ++dc) {
        if (d == 1 && dc == 0) continue;
        const int32_t cc = c + dc;
        if (cc < 0 || cc >= cols) continue;
        const uint32_t w = ((cc >> 5) == (c0 >> 5)) ? words[d][0] : words[d][1];
        any |= ((w >> (cc & 31)) & 1u) != 0;
      }
    }
    return any;
  }
};

// The bytes of an entry's crossing offsets: 0..sph-1 the offset in the hour
// at which that axis reaches its neighbour's centre, kOpen an open axis with
// no crossing this hour, kNone a closed axis (message sent, or the neighbour
// was not Available when the axis was set up)
constexpr uint32_t kOpen = 0xFEu;

// the open axes of an entry (bytes that are not kNone) as an 8-bit mask
__device__ __forceinline__ uint32_t open_axes(uint64_t c8) {
  const uint32_t closed = byte_lsbs(__vcmpeq4((uint32_t)c8, 0xFFFFFFFFu)) |
                          (byte_lsbs(__vcmpeq4((uint32_t)(c8 >> 32), 0xFFFFFFFFu)) << 4);
  return ~closed & 0xFFu;
}

// the axes of an entry crossing at offset o as an 8-bit mask (bytewise compares)
__device__ __forceinline__ uint32_t axes_at(uint64_t c8, uint32_t o) {
  const uint32_t oo = o * 0x01010101u;
  return byte_lsbs(__vcmpeq4((uint32_t)c8, oo)) | (byte_lsbs(__vcmpeq4((uint32_t)(c8 >> 32), oo)) << 4);
}

// One warp per replica; replicas come from a work list of (simulation,
// replica) items that every warp pulls from.  There is no CTA barrier: the
// warp's counters stay in registers, appends to the burning list are placed
// by ballot + popc, and phases are ordered with __syncwarp.  Per replica: an
// Available plane (burnable, not harvested, not yet ignited -- an ignition is
// one atomicAnd, whose old value also picks the single winner) and a Burned
// plane; with WIN their window around the ignition cell and the burning-list
// arrays sit in shared memory.  The scar plane (burnable and no longer
// Available) is written at the end.
//
// Each hour the burning cells' crossings are kept in a calendar: one linked
// list of list entries per crossing offset (an entry sits in the list of its
// earliest crossing) and a 64-bit mask of the offsets whose lists are not
// empty.  The next fire period to visit is the mask's lowest bit, and a
// visited period walks only the entries that cross in it.  Work is laid out
// one lane per cell, the 8 axes of a cell as independent chains in its lane:
// at the hour boundary (every listed cell) and for the cells ignited in a
// visited period.
template <int WPC, bool WIN, bool LAZY, bool PROF>
__device__ __forceinline__ void frontier_warp(const FrontierArgs &A) {
  // list links: 16 bits in shared memory (capacities there stay far below 2^16)
  using Link = typename std::conditional<WIN, uint16_t, int32_t>::type;
  constexpr int32_t kNil = -1;
  extern __shared__ __align__(16) uint32_t s_dyn[];
  __shared__ SimJob s_job[WPC];
  constexpr uint32_t FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int k = lane & 7, grp = lane >> 3;   // new-cell set-up: lane k of group grp owns axis k
  const uint32_t lt = (1u << lane) - 1u;
  const size_t slot = (size_t)blockIdx.x * WPC + wib;
  const int32_t cap = A.cap;
  // compact the list within an hour once it holds more than this many entries
  const int32_t compact_at = (A.compact_at > 0 && A.compact_at < cap) ? A.compact_at : cap - cap / 4;
  const uint32_t wait_limit = A.wait_limit ? A.wait_limit : kChunkSpinLimit;
  uint32_t *my = s_dyn + (size_t)wib * A.smem_warp_words;   // [Available win][Burned win][lists]
  uint32_t *erc;     // row << 16 | col
  uint8_t *ecofs;    // 8 crossing-offset bytes per entry
  Link *elink;       // next entry in the same calendar list
  Planes<WIN> pl;
  pl.gav = A.avail_scratch + slot * (size_t)A.pw_max;
  pl.gbr = A.brn_scratch + slot * (size_t)A.pw_max;
  if constexpr (WIN) {
    pl.sav = my;
    pl.sbr = my + kWinRows * kWinWords;
    uint32_t *ls = my + 2 * kWinRows * kWinWords;
    erc = ls;
    ecofs = reinterpret_cast<uint8_t *>(ls + cap);
    elink = reinterpret_cast<Link *>(ls + 3 * (size_t)cap);
  } else {
    pl.sav = pl.sbr = nullptr;
    erc = reinterpret_cast<uint32_t *>(A.ent_cell) + slot * cap;
    ecofs = A.ent_cofs + slot * (size_t)cap * 8;
    elink = reinterpret_cast<Link *>(A.ent_link) + slot * cap;
  }
  int64_t *eP = A.ent_P + slot * (size_t)cap * 8;
  __shared__ int32_t s_hits[WPC][32];                  // one round of crossing entries
  __shared__ int32_t s_head[WPC][64];                  // calendar: first entry per offset
  __shared__ uint32_t s_dbits[WPC][LAZY ? kWinRows * kWinWords / 32 : 1];   // chunks known done this hour
  __shared__ int32_t s_claim[WPC][LAZY ? 32 : 1];
  __shared__ long long s_prof[WPC][PROF ? kProfCounters : 1];
  int32_t *hitbuf = s_hits[wib];
  int32_t *head = s_head[wib];
  uint32_t *dbits = s_dbits[wib];
  int32_t *claim = s_claim[wib];
  SimJob &J = s_job[wib];

  for (;;) {
    long long item = -1;
    int32_t jidx = 0;
    if (lane == 0) {
      const unsigned long long i = atomicAdd(A.counter, 1ull);
      if ((int64_t)i < A.n_items) {
        item = A.item_list ? A.item_list[i] : (long long)i;
        jidx = (int32_t)find_job(A.item_begin, A.n_jobs, item);
        J = A.jobs[jidx];
        if (J.n_scen > 1) {   // this replica's scenario: its stacked table
          const int64_t s = J.scen[item - A.item_begin[jidx]];
          const int64_t n = (int64_t)J.rows * J.cols;
          J.base += s * J.scen_hours * n * 8;
          J.hros += s * J.scen_hours * n;
          J.hour += s * J.prep_hours;
          if (J.chunk_state) J.chunk_state += s * J.scen_hours * J.rows * J.wpr;
        }
      }
    }
    item = __shfl_sync(FULL, item, 0);
    jidx = __shfl_sync(FULL, jidx, 0);
    __syncwarp();
    if (item < 0) return;
    const unsigned long long t_start = A.trace.rec ? global_ns() : 0ull;
    const int32_t r = (int32_t)(item - A.item_begin[jidx]);
    const int32_t rows = J.rows, cols = J.cols, wpr = J.wpr;
    const int64_t n = (int64_t)rows * cols;
    const int32_t pw = rows * wpr;
    const int32_t sph = J.sph, H = J.hours;
    // A5 general condition (1): burning hours per day, drawn per replica
    int32_t bhours = 24;
    if (J.burn_max > 0) {
      const U4 x = philox4x32_10(U4{(uint32_t)r, 0u, 0u, 3u}, (uint32_t)J.seed, (uint32_t)(J.seed >> 32));
      bhours = J.burn_min + (int32_t)(((uint64_t)x.x * (uint64_t)(J.burn_max - J.burn_min + 1)) >> 32);
    }
    const bool lazy = LAZY && J.chunk_state != nullptr;
    const double delta = J.delta;
    const bool use_delta = delta > 0.0;   // A5 (i) burn-out on
    const uint64_t seed = J.seed;
    const float sigma = J.sigma;
    const uint32_t *burnable = J.burnable;
    int32_t *istep = J.ign_step ? J.ign_step + (size_t)r * n : nullptr;
    const int64_t dk = (k & 1) ? J.d_diag : J.d_orth;   // this lane's axis length
    const int32_t ic = J.ign_cell[r];
    // an ignition cell outside the grid or not burnable (possible only for
    // ignition cells a caller passes in): status 3, nothing else is written
    if ((uint32_t)ic >= (uint32_t)n ||
        !((__ldg(&burnable[(ic / cols) * wpr + ((ic % cols) >> 5)]) >> ((ic % cols) & 31)) & 1u)) {
      if (lane == 0) J.status[r] = 3;
      __syncwarp();
      continue;
    }
    const int32_t ir = ic / cols, icc = ic - ir * cols;
    // window of the done-chunk bitmap, centred on the ignition cell like the planes'
    const int32_t dr0 = min(max(ir - kWinRows / 2, 0), max(rows - kWinRows, 0));
    const int32_t dw0 = min(max((icc >> 5) - kWinWords / 2, 0), max(wpr - kWinWords, 0));
    pl.wpr = wpr;
    bool need_global = true;
    if constexpr (WIN) {   // window centred on the ignition cell, clamped to the grid
      pl.r0 = min(max(ir - kWinRows / 2, 0), max(rows - kWinRows, 0));
      pl.w0 = min(max((icc >> 5) - kWinWords / 2, 0), max(wpr - kWinWords, 0));
      need_global = rows > kWinRows || wpr > kWinWords;
      for (int32_t i = lane; i < kWinRows * kWinWords; i += 32) {
        const int32_t rr = pl.r0 + i / kWinWords, ww = pl.w0 + i % kWinWords;
        const uint32_t b = (rr < rows && ww < wpr) ? __ldg(&burnable[rr * wpr + ww]) : 0u;
        pl.sav[i] = b;
        pl.sbr[i] = ~b;   // cells that never burn count as Burned already
      }
    }
    if (need_global)
      for (int32_t i = lane; i < pw; i += 32) {
        const uint32_t b = __ldg(&burnable[i]);
        pl.gav[i] = b;
        pl.gbr[i] = ~b;
      }
    __syncwarp();

    // per-replica profile (J.prof, off unless the caller asked for it; the
    // layout of c2f_get_replica_profile): cycles in all, at hour boundaries,
    // finding + sending crossings and receiving (A), new-cell set-up (C);
    // visited periods, crossing entries, new cells, longest list; cycles of
    // (A) spent walking the period's calendar list, compactions within an
    // hour, rounds of crossing entries, new-cell passes (32 cells each)
    // (kept in shared memory, lane 0 only, so that they cost no registers)
    const bool prof = PROF && J.prof != nullptr;   // compiled out of the production kernels
    long long pc_t = 0;
    long long *pq = s_prof[wib];
    if (prof && lane == 0) {
#pragma unroll
      for (int i = 0; i < kProfCounters; ++i) pq[i] = 0;
      pq[0] = clock64();
    }

    // Step 1 of Alg. 1: the ignition cell burns from period 0
    int32_t live = 1, nign = 1, cnt = 1, status = 0;
    long long W = 0, s_done = 0;
    {
      if (lane == 0) {
        pl.take(ir, icc);
        if (istep) istep[ic] = 0;
      }
      __syncwarp();
      const uint32_t am = pl.avail_mask(rows, cols, ir, icc);
      if (lane < 8) {
        eP[lane] = 0;
        ecofs[lane] = (uint8_t)(((am >> lane) & 1u) ? kOpen : kNone);
      }
      if (lane == 0) erc[0] = rc_pack(ir, icc);
      if (am == 0) {   // no Available neighbour: Burned at the end of period 1
        if (lane == 0) pl.burn(ir, icc);
        live = 0;
        W = (H * sph >= 1) ? 1 : 0;
      }
      __syncwarp();
    }

    // On-demand table rows (lazy tables): before a row of hour h is read, the
    // chunk holding it must be done.  `slots` bit 0 asks for the cell's own
    // chunk, bit 1 + k for the chunk of its neighbour on axis k.  A chunk is
    // looked up in the bitmap of chunks known done this hour, else in
    // chunk_state: claimed when empty (the warp computes its claims at once,
    // all lanes on one chunk), waited for when another warp is computing it --
    // that warp is running and never waits while it holds a claim.
    auto ensure = [&](int32_t h, bool valid, int32_t cr, int32_t cc, uint32_t slots) {
      if (status != 0) return;   // the replica has stopped: no more claims or waits
      if (!valid) slots = 0;
      uint32_t todo = __reduce_or_sync(FULL, slots);
      uint32_t *sth = J.chunk_state + (size_t)h * pw;
      while (todo) {
        const int q = __ffs(todo) - 1;
        todo &= todo - 1;
        int32_t wr = -1, wc = 0;
        if ((slots >> q) & 1u) {
          int32_t nr = cr, nc = cc;
          if (q > 0) { nr += axis_dr(q - 1); nc += axis_dc(q - 1); }
          if (nr >= 0 && nr < rows && nc >= 0 && nc < cols) { wr = nr; wc = nc >> 5; }
        }
        const int32_t w = wr * wpr + wc;
        const bool inwin = wr >= dr0 && wr < dr0 + kWinRows && wc >= dw0 && wc < dw0 + kWinWords;
        const int32_t bi = inwin ? (wr - dr0) * kWinWords + (wc - dw0) : 0;
        bool need = false, mine = false;
        if (wr >= 0 && !(inwin && ((dbits[bi >> 5] >> (bi & 31)) & 1u))) {
          uint32_t st = ld_state(sth + w);
          if (st == 0u) {
            st = atomicCAS(sth + w, 0u, 1u);
            mine = st == 0u;
          }
          need = !mine && st < 2u;
          if (st >= 2u && inwin) atomicOr(&dbits[bi >> 5], 1u << (bi & 31));
        }
        const uint32_t mb = __ballot_sync(FULL, mine);
        if (mine) claim[__popc(mb & lt)] = w;
        __syncwarp();
        const int nm = __popc(mb);
        for (int i = 0; i < nm; ++i) table_chunk(J, h, claim[i]);
        if (mine && inwin) atomicOr(&dbits[bi >> 5], 1u << (bi & 31));
        if (need) {
          uint32_t polls = 0;
          bool gave_up = false;
          while (ld_state(sth + w) < 2u) {
            if (++polls > wait_limit) { status = 4; gave_up = true; break; }
            __nanosleep(128);
          }
          if (!gave_up && inwin) atomicOr(&dbits[bi >> 5], 1u << (bi & 31));
        }
        __syncwarp();
      }
      status = (int32_t)__reduce_max_sync(FULL, (uint32_t)status);   // the warp's worst status
    };

    // calendar: puts entry e into the list of offset nx; returns nx's bit
    // (0 when the entry has no crossing left this hour)
    auto push = [&](int32_t e, uint32_t nx) -> uint64_t {
      if (nx >= (uint32_t)sph) return 0ull;
      elink[e] = (Link)atom_exch_shared(&head[nx], e);
      return 1ull << nx;
    };
    auto cal_or = [&](uint64_t bits) -> uint64_t {   // OR of the lanes' calendar bits
      return ((uint64_t)__reduce_or_sync(FULL, (uint32_t)(bits >> 32)) << 32) |
             (uint64_t)__reduce_or_sync(FULL, (uint32_t)bits);
    };

    // drop Burned cells and cells with no open axis from the burning list
    // (order kept) when it nears its capacity within an hour, and rebuild the
    // calendar lists of the offsets from o on; returns the new calendar mask
    auto compact = [&](int32_t &count, uint32_t o) -> uint64_t {
      for (int32_t i = lane; i < 64; i += 32) head[i] = kNil;
      __syncwarp();
      int32_t out = 0;
      uint64_t cal = 0;
      for (int32_t b0 = 0; b0 < count; b0 += 32) {
        const int32_t e = b0 + lane;
        bool keep = false;
        uint32_t rc = 0;
        uint64_t c8 = ~0ull;
        int64_t P[8];
        if (e < count) {
          rc = erc[e];
          c8 = *reinterpret_cast<const uint64_t *>(ecofs + (size_t)e * 8);
          keep = open_axes(c8) != 0 && !pl.burned((int32_t)(rc >> 16), (int32_t)(rc & 0xFFFFu));
          if (keep) {
#pragma unroll
            for (int q = 0; q < 8; ++q) P[q] = eP[(size_t)e * 8 + q];
          }
        }
        const uint32_t bal = __ballot_sync(FULL, keep);
        const int32_t pos = out + __popc(bal & lt);
        __syncwarp();
        uint64_t bit = 0;
        if (keep) {
          erc[pos] = rc;
          *reinterpret_cast<uint64_t *>(ecofs + (size_t)pos * 8) = c8;
#pragma unroll
          for (int q = 0; q < 8; ++q) eP[(size_t)pos * 8 + q] = P[q];
          const uint32_t nx = min_byte8(c8);
          if (nx >= o) bit = push(pos, nx);
        }
        cal |= cal_or(bit);
        out += __popc(bal);
        __syncwarp();
      }
      count = out;
      return cal;
    };

    for (int32_t h = 0; h < H && live > 0 && status == 0; ++h) {
      const int32_t s0 = h * sph + 1, L = s0 + sph - 1;
      if (h % 24 >= bhours) {   // a dormant hour: nothing moves, no work is counted
        s_done = L;
        continue;
      }
      const int64_t *baseh = J.base + (size_t)h * n * 8;
      const double *hrosh = J.hros + (size_t)h * n;
      // receive tests can be skipped when the threshold is 0 and every HROS of
      // the hour is positive (then HROS * f > 0), or when the threshold is < 0
      const bool gate_free = J.recv_gate <= 1 || (J.recv_gate == 2 && J.hour && J.hour[h].pos);
      int32_t burned = 0;   // cells Burned at the end of the period being visited
      if (lazy) {
        for (int32_t i = lane; i < kWinRows * kWinWords / 32; i += 32) dbits[i] = 0u;
      }
      for (int32_t i = lane; i < 64; i += 32) head[i] = kNil;
      __syncwarp();
      uint64_t cal = 0;   // offsets of this hour whose calendar list is not empty

      if (prof && lane == 0) pc_t = clock64();
      // ---- hour boundary, one lane per listed cell, 32 cells at a time:
      // (i) drop Burned cells and cells with no open axis (order kept);
      // (ii) the cell's perturbation for this hour; (iii) on every open axis,
      // the crossing period of this hour, or the progress carried to the next;
      // (iv) the cell into the calendar list of its first crossing.
      {
        int32_t out = 0;
        for (int32_t b0 = 0; b0 < cnt; b0 += 32) {
          const int32_t e = b0 + lane;
          bool keep = false;
          uint32_t rc = 0u, m = 0u;
          if (e < cnt) {
            rc = erc[e];
            m = open_axes(*reinterpret_cast<const uint64_t *>(ecofs + (size_t)e * 8));
            keep = m != 0u && !pl.burned((int32_t)(rc >> 16), (int32_t)(rc & 0xFFFFu));
          }
          const int32_t cr = (int32_t)(rc >> 16), cc = (int32_t)(rc & 0xFFFFu);
          if (lazy) ensure(h, keep, cr, cc, 1u);   // this hour's row of the cell
          const int64_t cell = (int64_t)cr * cols + cc;
          int64_t P[8], bk[8];
          if (keep) {   // progress and rate row: 64 bytes each, four 16-byte loads
            const longlong2 *pp = reinterpret_cast<const longlong2 *>(eP + (size_t)e * 8);
            const longlong2 *rw = reinterpret_cast<const longlong2 *>(baseh + cell * 8);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const longlong2 a = pp[j], b = __ldcg(rw + j);
              P[2 * j] = a.x; P[2 * j + 1] = a.y;
              bk[2 * j] = b.x; bk[2 * j + 1] = b.y;
            }
            // the cell's row of the next hour into L2, for the next boundary
            if (!LAZY && h + 1 < H) prefetch_l2(baseh + n * 8 + cell * 8);
          } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) P[q] = bk[q] = 0;
          }
          const float f = keep ? noise_factor(seed, (uint32_t)r, (uint32_t)cell, (uint32_t)h, sigma) : 1.0f;
          const uint64_t F = noise_fixed(f);
          // A5 (i): a cell whose HROS * f is below delta still sends in the
          // first period of the hour and is Burned after it
          const bool dies = keep && use_delta && below_delta(hrosh, cell, f, delta);
          uint64_t c8 = ~0ull;   // crossing-offset bytes
          const uint32_t am = keep ? (m & pl.avail_mask(rows, cols, cr, cc)) : 0u;   // open axes toward Available cells
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            uint32_t cof = kNone;
            if ((am >> q) & 1u) {
              const int64_t dq = (q & 1) ? J.d_diag : J.d_orth;
              const int64_t inc = apply_noise(bk[q], F, dq);
              const int64_t rem = dq - P[q];
              if (inc > 0 && inc * sph >= rem) {
                cof = (uint32_t)(ceil_div_small(rem, inc) - 1);
              } else {
                P[q] += inc * sph;
                cof = kOpen;
              }
              if (dies && cof != 0u) cof = kNone;
            }
            c8 = (c8 & ~(0xFFull << (8 * q))) | ((uint64_t)cof << (8 * q));
          }
          const bool dying = dies && pl.burn(cr, cc);
          const uint32_t bal = __ballot_sync(FULL, keep);
          const int32_t pos = out + __popc(bal & lt);
          __syncwarp();   // every lane has read its entry before any slot is rewritten
          uint64_t bit = 0;
          if (keep) {
            erc[pos] = rc;
            *reinterpret_cast<uint64_t *>(ecofs + (size_t)pos * 8) = c8;
            longlong2 *pp = reinterpret_cast<longlong2 *>(eP + (size_t)pos * 8);
#pragma unroll
            for (int j = 0; j < 4; ++j) pp[j] = make_longlong2(P[2 * j], P[2 * j + 1]);
            bit = push(pos, min_byte8(c8));
          }
          cal |= cal_or(bit);
          out += __popc(bal);
          burned += __popc(__ballot_sync(FULL, dying));
          __syncwarp();
        }
        cnt = out;
      }
      if (prof && lane == 0) pq[1] += clock64() - pc_t;
      if (status) break;
      // cells that die this hour (A5 (i)) are Burned at the end of its first
      // period: that period is visited even if no axis crosses in it
      if (burned) cal |= 1ull;

      // ---- periods of this hour at which some axis reaches a centre
      while (cal != 0ull) {
        const uint32_t o = (uint32_t)(__ffsll((long long)cal) - 1);
        const int32_t s = s0 + (int32_t)o;
        W += (long long)live * (long long)(s - s_done);
        s_done = s;
        if (prof && lane == 0) { pc_t = clock64(); pq[4] += 1; pq[7] = max(pq[7], (long long)cnt); }
        if (cnt > compact_at) {   // keep room for new cells
          cal = compact(cnt, o);
          if (prof && lane == 0) pq[9] += 1;
        }
        cal &= ~(1ull << o);
        int32_t nnew = cnt;
        bool ovf = false;
        // (A) send and receive: the entries of offset o's calendar list, 32 at
        // a time (lane 0 walks the list); each lane takes one entry: every
        // axis crossing at o is handled in turn (target tested, ignited,
        // appended by ballot + popc), then the entry goes into the list of its
        // next crossing
        int32_t cur = head[o];
        int32_t walked = 0;   // a list holds each entry at most once: never more than cnt
        while (cur != kNil) {
          long long pw0 = 0;
          if (prof && lane == 0) pw0 = clock64();
          int32_t take_n = 0;
          if (lane == 0) {
            while (cur != kNil && take_n < 32) {
              hitbuf[take_n++] = cur;
              cur = elink[cur];
              if (cur == (int32_t)(Link)kNil) cur = kNil;
            }
          }
          take_n = __shfl_sync(FULL, take_n, 0);
          cur = __shfl_sync(FULL, cur, 0);
          __syncwarp();
          walked += take_n;
          if (walked > cnt) { status = 2; break; }   // cannot happen; a broken list stops here
          if (prof && lane == 0) { pq[8] += clock64() - pw0; pq[5] += take_n; pq[10] += 1; }
          const int32_t ent = lane < take_n ? hitbuf[lane] : -1;
          uint64_t cof8 = ~0ull;
          uint32_t rc = 0;
          if (ent >= 0) {
            cof8 = *reinterpret_cast<const uint64_t *>(ecofs + (size_t)ent * 8);
            rc = erc[ent];
          }
          const uint32_t cm = ent >= 0 ? axes_at(cof8, o) : 0u;   // axes crossing at o
          const int32_t cr = (int32_t)(rc >> 16), cc = (int32_t)(rc & 0xFFFFu);
          if (lazy && !gate_free) ensure(h, ent >= 0, cr, cc, cm << 1);   // receivers' HROS
          uint32_t todo = cm;
          const int rounds = (int)__reduce_max_sync(FULL, (uint32_t)__popc(cm));
          for (int it2 = 0; it2 < rounds; ++it2) {
            bool won = false;
            uint32_t wrc = 0;
            int64_t jc = 0;
            if (todo) {
              const int q = __ffs(todo) - 1;
              todo &= todo - 1;
              const int32_t nr = cr + axis_dr(q), nc = cc + axis_dc(q);
              jc = (int64_t)nr * cols + nc;
              wrc = rc_pack(nr, nc);
              if (gate_free) {
                won = pl.take(nr, nc);   // taken iff it was Available; one atomic decides
              } else if (pl.avail(nr, nc) && receive_ok(J, r, jc, h, n)) {   // else consumed
                won = pl.take(nr, nc);
              }
            }
            const uint32_t wins = __ballot_sync(FULL, won);
            if (won) {
              const int32_t idx = nnew + __popc(wins & lt);
              if (idx < cap) erc[idx] = wrc; else ovf = true;
              if (istep) istep[jc] = s;
              // the new cell's table row, read when it is set up: into L1 when
              // the table is complete (read-only here), else into L2
              if (LAZY) prefetch_l2(baseh + jc * 8);
              else prefetch_row_l1(baseh + jc * 8);
            }
            nnew += __popc(wins);
          }
          uint64_t bit = 0;
          if (ent >= 0) {   // the axes that crossed close; the entry moves to its next crossing
            uint64_t nc8 = cof8;
#pragma unroll
            for (int q = 0; q < 8; ++q)
              if ((cm >> q) & 1u) nc8 |= 0xFFull << (8 * q);
            *reinterpret_cast<uint64_t *>(ecofs + (size_t)ent * 8) = nc8;
            bit = push(ent, min_byte8(nc8));
          }
          cal |= cal_or(bit);
          __syncwarp();
        }
        if (prof && lane == 0) {
          const long long t1 = clock64();
          pq[2] += t1 - pc_t;
          pc_t = t1;
          pq[6] += nnew - cnt;
        }
        if (status) break;
        if (__any_sync(FULL, ovf)) { status = 1; break; }
        __syncwarp();
        // (C) cells ignited in period s, four at a time, lane k of each 8-lane
        // group owning axis k: open axes, first crossings, progress to the end
        // of the hour, burn-out tests, and the cell into the calendar
        if (lazy) {   // this hour's rows of the new cells
          for (int32_t b0 = cnt; b0 < nnew; b0 += 32) {
            const int32_t e = b0 + lane;
            const uint32_t rc = e < nnew ? erc[e] : 0u;
            ensure(h, e < nnew, (int32_t)(rc >> 16), (int32_t)(rc & 0xFFFFu), 1u);
          }
          if (status) break;
        }
        for (int32_t b0 = cnt; b0 < nnew; b0 += 4) {
          if (prof && lane == 0) pq[11] += 1;
          const int32_t e = b0 + grp;
          const bool act = e < nnew;
          const uint32_t rc = act ? erc[e] : 0u;
          const int32_t cr = (int32_t)(rc >> 16), cc = (int32_t)(rc & 0xFFFFu);
          const int64_t cell = (int64_t)cr * cols + cc;
          const int32_t nr = cr + axis_dr(k), nc = cc + axis_dc(k);
          const bool ingrid = act && nr >= 0 && nr < rows && nc >= 0 && nc < cols;
          // the table load issued early; through L1 (the row was prefetched
          // there) unless other warps may be writing the table (lazy rows)
          const int64_t bk = act ? (LAZY ? __ldcg(baseh + cell * 8 + k) : __ldca(baseh + cell * 8 + k)) : 0;
          const bool open = ingrid && pl.avail(nr, nc);
          // the perturbation does not depend on the loads above: computed while they are in flight
          const float f = act ? noise_factor(seed, (uint32_t)r, (uint32_t)cell, (uint32_t)h, sigma) : 1.0f;
          const bool ignq = ingrid && !open;   // ignited, or never burnable (pre-marked Burned)
          const uint32_t omask = group_bits(open);
          uint32_t mask = omask;
          bool dies = false;
          if (act && use_delta) {
            if (below_delta(hrosh, cell, f, delta)) { dies = true; mask = 0; }   // A5 (i)
          }
          uint32_t cof = ((mask >> k) & 1u) ? kOpen : kNone;
          int64_t P = 0;
          if (act && ((mask >> k) & 1u) && s < L) {
            const int32_t nmax = L - s;   // periods left in the hour
            const int64_t inc = apply_noise(bk, noise_fixed(f), dk);
            if (inc > 0 && inc * nmax >= dk) cof = o + (uint32_t)ceil_div_small(dk, inc);
            else P = inc * nmax;
          }
          const uint32_t nx = group_min(cof);
          uint32_t newly = 0;   // cells this lane turned Burned (its own cell, its axis neighbour)
          uint64_t bit = 0;
          if (act) {
            ecofs[(size_t)e * 8 + k] = (uint8_t)cof;
            eP[(size_t)e * 8 + k] = P;
            if (k == 0) {
              bit = push(e, nx);
              if (omask == 0 || dies)   // this cell: A5 (ii) no Available neighbour, or (i)
                newly += pl.burn(cr, cc) ? 1u : 0u;
            }
            // A5 (ii) for the ignited neighbour on this lane's axis
            if (ignq && !pl.any_avail_nbr(rows, cols, nr, nc)) newly += pl.burn(nr, nc) ? 1u : 0u;
          }
          cal |= cal_or(bit);
          burned += (int32_t)__reduce_add_sync(FULL, newly);
        }
        __syncwarp();
        if (prof && lane == 0) pq[3] += clock64() - pc_t;
        // every crossing pushed in this period lies after it; a bit at or
        // before o cannot happen and would revisit a period
        if (cal & ((2ull << o) - 1ull)) { status = 2; break; }
        const int32_t added = nnew - cnt;
        nign += added;
        live += added - burned;
        burned = 0;
        cnt = nnew;
        if (live == 0) break;
      }
      if (status == 0) { W += (long long)live * (long long)(L - s_done); s_done = L; }
    }
    {   // scar plane: burnable cells that are no longer Available
      uint32_t *dst = J.ign_plane + (size_t)r * pw;
      for (int32_t i = lane; i < pw; i += 32) {
        const int32_t rr = i / wpr, ww = i - rr * wpr;
        uint32_t a;
        if (pl.in_win(rr, ww)) a = pl.sav[(rr - pl.r0) * kWinWords + (ww - pl.w0)];
        else a = pl.gav[i];
        dst[i] = __ldg(&burnable[i]) & ~a;
      }
    }
    if (lane == 0) {
      if (A.trace.rec) trace_record(A.trace, kTraceReplica, (uint32_t)r, J.trace_tag, t_start, global_ns());
      J.work[r] = W;
      J.n_ignited[r] = nign;
      J.status[r] = status;
      if (prof) {
        long long *q = J.prof + (size_t)r * kProfCounters;
        q[0] = clock64() - pq[0];
#pragma unroll
        for (int i = 1; i < kProfCounters; ++i) q[i] = pq[i];
      }
    }
    __syncwarp();
  }
}

// Variants: warps per CTA (1, 2, 4); planes windowed and lists in shared
// memory (w), or everything in global memory (g); l: tables filled on demand;
// p: the per-replica profile counters compiled in (one-warp CTAs; the
// production kernels leave that code out, which makes them about 4 % faster).
// Register budgets: one-warp CTAs sized so that 11 fit on an SM (the
// pipelined steps run the next table build beside the frontier, which more
// registers a thread would crowd out; fewer would spill); two-warp CTAs so
// that 5 fit
__global__ void __launch_bounds__(32, 11) k_frontier_g1(FrontierArgs A) { frontier_warp<1, false, false, false>(A); }
__global__ void __launch_bounds__(64, 5) k_frontier_g2(FrontierArgs A) { frontier_warp<2, false, false, false>(A); }
__global__ void __launch_bounds__(128) k_frontier_g4(FrontierArgs A) { frontier_warp<4, false, false, false>(A); }
__global__ void __launch_bounds__(32, 11) k_frontier_w1(FrontierArgs A) { frontier_warp<1, true, false, false>(A); }
__global__ void __launch_bounds__(64, 5) k_frontier_w2(FrontierArgs A) { frontier_warp<2, true, false, false>(A); }
__global__ void __launch_bounds__(128) k_frontier_w4(FrontierArgs A) { frontier_warp<4, true, false, false>(A); }
__global__ void __launch_bounds__(32, 11) k_frontier_pg1(FrontierArgs A) { frontier_warp<1, false, false, true>(A); }
__global__ void __launch_bounds__(32, 11) k_frontier_pw1(FrontierArgs A) { frontier_warp<1, true, false, true>(A); }
// on-demand table rows: one warp per CTA; the FBP code inlined into the
// frontier needs the whole register budget of a one-warp CTA
__global__ void __launch_bounds__(32, 1) k_frontier_lg1(FrontierArgs A) { frontier_warp<1, false, true, false>(A); }
__global__ void __launch_bounds__(32, 1) k_frontier_lw1(FrontierArgs A) { frontier_warp<1, true, true, false>(A); }
__global__ void __launch_bounds__(32, 1) k_frontier_plg1(FrontierArgs A) { frontier_warp<1, false, true, true>(A); }
__global__ void __launch_bounds__(32, 1) k_frontier_plw1(FrontierArgs A) { frontier_warp<1, true, true, true>(A); }

// ------------------------------------------------------------------ K4
// counts[c] = sum over replicas of the scar bit of c.  Each thread owns one
// 32-cell word and adds the replicas' words into a bit-sliced (vertical)
// counter: plane i holds bit i of the 32 per-cell counts.
// With scen, only the replicas whose drawn weather scenario is `want` count.
__global__ void k_burn_prob(const uint32_t *__restrict__ planes, int32_t R, int32_t rows,
                            int32_t cols, int32_t wpr, int32_t r_chunk, uint32_t *counts,
                            int32_t accumulate, const int32_t *__restrict__ scen, int32_t want) {
  const int64_t pw = (int64_t)rows * wpr;
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= pw) return;
  const int32_t r0 = blockIdx.y * r_chunk;
  const int32_t r1 = min(R, r0 + r_chunk);
  uint32_t c[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) c[i] = 0;
  for (int32_t r = r0; r < r1; ++r) {
    if (scen && __ldg(&scen[r]) != want) continue;
    uint32_t carry = __ldg(&planes[(size_t)r * pw + w]);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const uint32_t t = c[i] & carry;
      c[i] ^= carry;
      carry = t;
    }
  }
  const int32_t row = (int32_t)(w / wpr), cw = (int32_t)(w % wpr);
  for (int b = 0; b < 32; ++b) {
    const int32_t col = cw * 32 + b;
    if (col >= cols) break;
    uint32_t v = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) v |= ((c[i] >> b) & 1u) << i;
    const int64_t cell = (int64_t)row * cols + col;
    if (accumulate) { if (v) atomicAdd(&counts[cell], v); }
    else counts[cell] = v;
  }
}

// ignition steps -> one byte per (replica, cell): ignited by period smax
__global__ void k_scar_at_step(const int32_t *__restrict__ ign_step, int64_t total, int32_t smax,
                               uint8_t *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int32_t s = ign_step[i];
  out[i] = (s >= 0 && s <= smax) ? 1 : 0;
}

// scar bits -> one byte per (replica, cell)
__global__ void k_scar_bytes(const uint32_t *__restrict__ planes, int32_t R, int32_t rows,
                             int32_t cols, int32_t wpr, uint8_t *out) {
  const int64_t n = (int64_t)rows * cols;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * R) return;
  const int64_t r = i / n, cell = i % n;
  const int32_t row = (int32_t)(cell / cols), col = (int32_t)(cell % cols);
  out[i] = (planes[(size_t)r * rows * wpr + (size_t)row * wpr + (col >> 5)] >> (col & 31)) & 1u;
}

// ------------------------------------------------------------------ calibration
// FP64 fused multiply-add throughput of the device: eight independent chains
// per thread, enough warps to cover the pipe's latency; the roofline peak of
// the table kernel, which is FP64-bound.
__global__ void k_dfma_peak(double *out, int32_t iters) {
  const double m = 0.999999999, c = 1e-12;
  double a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  for (int32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = __fma_rn(a[j], m, c);
  }
  double t = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) t += a[j];
  if (t == 12345.678) out[blockIdx.x] = t;   // never true; keeps the chains alive
}

// ------------------------------------------------------------------ scar comparison
// Sec. 4.1 compares two runs' scars X^t, Y^t (0-1 grids, 1 = ignited by the
// end of weather hour t) by MSE, SSIM and, for the final scars, ||X - Y||.
// For 0-1 grids all three are functions of a = |X|, b = |Y|, c = |X and Y|
// and N: sum |X - Y|^2 = a + b - 2c; the means are a/N, b/N; the 1/(N-1)
// variances a(N-a)/(N(N-1)), b(N-b)/(N(N-1)); the covariance
// (cN - ab)/(N(N-1)).  SSIM takes Wang et al.'s C1 = 0.01^2, C2 = 0.03^2
// (dynamic range 1) and sigma_X^2 + sigma_Y^2 + C2 in its denominator.
constexpr double kSsimC1 = 0.0001;   // (0.01 * 1)^2
constexpr double kSsimC2 = 0.0009;   // (0.03 * 1)^2

__device__ inline void scar_metrics(double a, double b, double c, double n, double *mse,
                                    double *ssim) {
  *mse = (a + b - 2.0 * c) / n;
  const double mx = a / n, my = b / n;
  const double nn1 = n * (n - 1.0);
  const double vx = a * (n - a) / nn1, vy = b * (n - b) / nn1;
  const double cxy = (c * n - a * b) / nn1;
  *ssim = ((2.0 * mx * my + kSsimC1) * (2.0 * cxy + kSsimC2)) /
          ((mx * mx + my * my + kSsimC1) * (vx + vy + kSsimC2));
}

// weather hour in which ignition step s falls (step 0 = the ignition, hour 0);
// -1 for a cell that never ignites
__device__ __forceinline__ int32_t ign_hour(int32_t s, int32_t sph) {
  return s < 0 ? -1 : (s == 0 ? 0 : (s - 1) / sph);
}

__device__ __forceinline__ void count_cell(int32_t sx, int32_t sy, int32_t sph, int32_t H,
                                           uint32_t *hist) {
  const int32_t hx = ign_hour(sx, sph), hy = ign_hour(sy, sph);
  if (hx >= 0 && hx < H) atomicAdd(&hist[hx], 1u);
  if (hy >= 0 && hy < H) atomicAdd(&hist[H + hy], 1u);
  if (hx >= 0 && hy >= 0 && max(hx, hy) < H) atomicAdd(&hist[2 * H + max(hx, hy)], 1u);
}

__device__ __forceinline__ void count_cells4(const int4 &a, const int4 &b, int32_t sph, int32_t H,
                                             uint32_t *hist) {
  // four cells that neither run ignites (the common case) cost one test
  if ((a.x & a.y & a.z & a.w & b.x & b.y & b.z & b.w) < 0) return;
  count_cell(a.x, b.x, sph, H, hist);
  count_cell(a.y, b.y, sph, H, hist);
  count_cell(a.z, b.z, sph, H, hist);
  count_cell(a.w, b.w, sph, H, hist);
}

// One CTA per replica: histograms of the ignition hours of X, of Y and of the
// later of the two (cells both runs ignite), then prefix sums over hours give
// a, b, c of every hour's scars; one pass over the two ignition-step arrays,
// streamed with 16-byte loads (when the rows are aligned), four per array in
// flight per thread.  128-thread CTAs so that every replica of a launch is
// resident at once.  Dynamic shared memory: 3 H counters.  The final scars are
// the scars of the last hour, so ||X - Y|| comes from the same counts.
__global__ void __launch_bounds__(128) k_compare_hours(const int32_t *__restrict__ step_x,
                                                       const int32_t *__restrict__ step_y, int64_t n,
                                                       int32_t sph, int32_t H, double *mse, double *ssim,
                                                       double *dnorm) {
  extern __shared__ uint32_t hist[];
  const int32_t r = blockIdx.x;
  for (int32_t i = threadIdx.x; i < 3 * H; i += blockDim.x) hist[i] = 0u;
  __syncthreads();
  const int32_t *x = step_x + (size_t)r * n;
  const int32_t *y = step_y + (size_t)r * n;
  if ((n & 3) == 0 && ((reinterpret_cast<uintptr_t>(step_x) | reinterpret_cast<uintptr_t>(step_y)) & 15u) == 0) {
    const int4 *x4 = reinterpret_cast<const int4 *>(x);
    const int4 *y4 = reinterpret_cast<const int4 *>(y);
    const int64_t n4 = n / 4, bd = blockDim.x;
    int64_t i = threadIdx.x;
    for (; i + 3 * bd < n4; i += 4 * bd) {
      int4 a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = __ldcs(x4 + i + u * bd);
        b[u] = __ldcs(y4 + i + u * bd);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) count_cells4(a[u], b[u], sph, H, hist);
    }
    for (; i < n4; i += bd) count_cells4(__ldcs(x4 + i), __ldcs(y4 + i), sph, H, hist);
  } else {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) count_cell(__ldcs(x + i), __ldcs(y + i), sph, H, hist);
  }
  __syncthreads();
  if (threadIdx.x < 3) {   // counts of scars at hour t: inclusive prefix sums
    uint32_t *h = hist + threadIdx.x * H;
    uint32_t acc = 0u;
    for (int32_t t = 0; t < H; ++t) { acc += h[t]; h[t] = acc; }
  }
  __syncthreads();
  for (int32_t t = threadIdx.x; t < H; t += blockDim.x) {
    double m, q;
    scar_metrics((double)hist[t], (double)hist[H + t], (double)hist[2 * H + t], (double)n, &m, &q);
    if (mse) mse[(size_t)r * H + t] = m;
    if (ssim) ssim[(size_t)r * H + t] = q;
  }
  if (dnorm && threadIdx.x == 0)   // |X xor Y| = a + b - 2c, exact in binary64
    dnorm[r] = sqrt((double)hist[H - 1] + (double)hist[2 * H - 1] - 2.0 * (double)hist[3 * H - 1]);
}

// ||X - Y|| of the final scars from the bit planes: one CTA per replica
// (256 threads), popcounts of X, Y and X and Y over the replica's words.
__global__ void k_compare_final(const uint32_t *__restrict__ px, const uint32_t *__restrict__ py,
                                int64_t pw, double *dnorm) {
  __shared__ unsigned long long part[8];
  const int32_t r = blockIdx.x;
  const uint32_t *x = px + (size_t)r * pw;
  const uint32_t *y = py + (size_t)r * pw;
  unsigned long long d = 0;   // sum |X - Y|^2 = |X xor Y|
  for (int64_t i = threadIdx.x; i < pw; i += blockDim.x) d += (unsigned)__popc(__ldcs(x + i) ^ __ldcs(y + i));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    dnorm[r] = sqrt((double)t);
  }
}

}  // namespace c2f
