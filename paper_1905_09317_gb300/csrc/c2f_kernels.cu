// c2f_kernels.cu -- the GB300 kernels of the fire-growth path.
//
//   k_cell_prep / k_hour_prep   hoisted per-cell and per-hour FBP terms
//   k_ros_table   (K1)  per (cell, hour): FBP HROS/BROS/LB, Eqs. (1)-(4), the 8
//                       axis rates as 2^32 fixed-point per-period increments
//   k_ignite      (K2)  Step 1 of Alg. 1: ignition cell per replica
//   k_frontier    (K3)  Step 2 of Alg. 1 for whole replicas: send / receive /
//                       burn-out per fire period, one CTA per replica
//   k_burn_prob   (K4)  burn-probability counts over replicas
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
  return e;
}

__device__ __constant__ int kDR[8] = {0, -1, -1, -1, 0, 1, 1, 1};
__device__ __constant__ int kDC[8] = {1, 1, 0, -1, -1, -1, 0, 1};

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

__global__ void __launch_bounds__(128) k_ros_table(RosTableArgs a) {
  const int64_t n = (int64_t)a.rows * a.cols;
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= n) return;
  const int h = a.hour0 + blockIdx.y;
  const int32_t row = (int32_t)(cell / a.cols), col = (int32_t)(cell % a.cols);
  const bool burn = (a.burnable[(int64_t)row * a.wpr + (col >> 5)] >> (col & 31)) & 1u;
  double ros[8];
  double hr = 0.0;
  if (!burn) {
#pragma unroll
    for (int k = 0; k < 8; ++k) ros[k] = 0.0;
  } else if (a.const_ros > 0.0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) ros[k] = a.const_ros;
    hr = a.const_ros;
  } else {
    const int fuel = a.fuel[cell];
    const double gs = a.slope ? (double)a.slope[cell] : 0.0;
    FbpOut o;
    fbp_row(fuel, gs, a.cell[cell], a.hour[h], a.pcf, a.ellipse_mode, &o);
#pragma unroll
    for (int k = 0; k < 8; ++k) ros[k] = o.ros[k];
    hr = o.hros;
  }
  const size_t idx = (size_t)h * n + cell;
  if (a.base) {
    longlong2 *dst = reinterpret_cast<longlong2 *>(a.base + idx * 8);
#pragma unroll
    for (int k = 0; k < 8; k += 2)
      dst[k / 2] = make_longlong2(fixed_of(__dmul_rn(ros[k], a.dt2p32)),
                                  fixed_of(__dmul_rn(ros[k + 1], a.dt2p32)));
  }
  if (a.hros) a.hros[idx] = hr;
  if (a.hros_pos && burn && !(hr > 1e-200)) atomicAnd(a.hros_pos, 0);
  if (a.ros8) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a.ros8[(size_t)cell * 8 + k] = ros[k];
  }
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
}

// ------------------------------------------------------------------ K3
__device__ __forceinline__ bool plane_bit(const uint32_t *p, int32_t wpr, int32_t r, int32_t c) {
  return (p[(int64_t)r * wpr + (c >> 5)] >> (c & 31)) & 1u;
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

// smallest n >= 1 with n * inc >= rem, given that it is at most a few dozen
__device__ __forceinline__ int32_t ceil_div_small(int64_t rem, int64_t inc) {
  const float q = __fdiv_rn((float)rem, (float)inc);
  int32_t n = (q < 4096.0f) ? (int32_t)ceilf(q) : 4096;
  if (n < 1) n = 1;
  while ((int64_t)n * inc < rem) ++n;
  while (n > 1 && (int64_t)(n - 1) * inc >= rem) --n;
  return n;
}

// receive test of a messaged Available cell (Sec. 3.1): HROS * f > threshold
__device__ inline bool receive_ok(const SimJob &J, int32_t r, int64_t j, int32_t h, int64_t n) {
  if (J.thr < 0.0) return true;
  const double hr = J.hros[(size_t)h * n + j];
  if (J.thr == 0.0) {
    if (hr > 1e-200) return true;   // f >= exp(-5.9) for sigma <= 1, so HROS * f > 0
    if (!(hr > 0.0)) return false;
  }
  const float f = noise_factor(J.seed, (uint32_t)r, (uint32_t)j, (uint32_t)h, J.sigma);
  return __dmul_rn(hr, (double)f) > J.thr;
}

// true if some neighbour of (r, c) is still Available (bit set in the
// Available plane: burnable, not harvested, not ignited)
__device__ inline bool has_available_nbr(const uint32_t *avail, int32_t wpr, int32_t rows,
                                         int32_t cols, int32_t r, int32_t c) {
  uint32_t words[3][2];
  const int32_t c0 = c > 0 ? c - 1 : 0, c1 = c + 1 < cols ? c + 1 : cols - 1;
  const int32_t w0 = c0 >> 5, w1 = c1 >> 5;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int32_t rr = r - 1 + d;
    const bool ok = rr >= 0 && rr < rows;
    words[d][0] = ok ? avail[(int64_t)rr * wpr + w0] : 0u;
    words[d][1] = ok ? avail[(int64_t)rr * wpr + w1] : 0u;
  }
  bool any = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int dc = -1; dc <= 1; ++dc) {
      if (d == 1 && dc == 0) continue;
      const int32_t cc = c + dc;
      if (cc < 0 || cc >= cols) continue;
      const uint32_t w = ((cc >> 5) == w0) ? words[d][0] : words[d][1];
      any |= ((w >> (cc & 31)) & 1u) != 0;
    }
  }
  return any;
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
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <int T>
struct FrontierShared {
  SimJob job;
  int64_t item;
  int32_t nnew, overflow, hros_pos;
  int32_t burn[2];
  uint32_t minnext[2];
  int32_t warp_tot[T / 32];
  int32_t out_base;
};

// min over the 8 lanes of this lane's group
__device__ __forceinline__ uint32_t group_min(uint32_t v) {
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// OR of a per-lane bit over the 8 lanes of this lane's group, as an 8-bit mask (bit k = lane k)
__device__ __forceinline__ uint32_t group_bits(bool b) {
  const uint32_t bal = __ballot_sync(0xffffffffu, b);
  return (bal >> (threadIdx.x & 24)) & 0xFFu;
}

// One CTA per replica, taken from a work list of (simulation, replica) items.
// Eight lanes cooperate on one burning cell, lane k owning axis k, so the
// per-axis work of a cell (crossing tests, increments, crossing periods,
// burn-out tests of the neighbour on that axis) runs side by side.  Each
// visited period costs two CTA barriers: sends + receives, then the set-up of
// the cells ignited in that period.  The replica's state is one Available
// bit plane (burnable and not yet ignited; an ignition is one atomicAnd that
// also tells the single winner) held in shared memory when it fits (SMEM) and
// in per-CTA global scratch otherwise, plus a Burned plane in global scratch;
// the scar plane is written out at the end.
template <int T, bool SMEM>
__device__ __forceinline__ void frontier_body(const FrontierArgs &A) {
  constexpr int G = T / 8;   // cell groups per CTA
  extern __shared__ __align__(16) uint32_t s_planes[];
  __shared__ FrontierShared<T> S;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = tid & 7, g = tid >> 3;
  const size_t slot = blockIdx.x;
  const int32_t cap = A.cap;
  int32_t *ecell = A.ent_cell + slot * cap;
  uint8_t *emask = A.ent_mask + slot * cap;
  uint8_t *enext = A.ent_next + slot * cap;
  uint8_t *ecofs = A.ent_cofs + slot * (size_t)cap * 8;
  int64_t *eP = A.ent_P + slot * (size_t)cap * 8;

  for (;;) {
    if (tid == 0) {
      const unsigned long long i = atomicAdd(A.counter, 1ull);
      int64_t item = -1;
      if ((int64_t)i < A.n_items) item = A.item_list ? A.item_list[i] : (int64_t)i;
      S.item = item;
      if (item >= 0) {
        S.job = A.jobs[find_job(A.item_begin, A.n_jobs, item)];
        S.hros_pos = S.job.hros_pos ? *S.job.hros_pos : 0;
      }
    }
    __syncthreads();
    const int64_t item = S.item;
    if (item < 0) return;
    const SimJob &J = S.job;
    const int32_t r = (int32_t)(item - A.item_begin[find_job(A.item_begin, A.n_jobs, item)]);
    const int32_t rows = J.rows, cols = J.cols, wpr = J.wpr;
    const int64_t n = (int64_t)rows * cols;
    const size_t pw = (size_t)rows * wpr;
    const bool gate_free = (J.thr < 0.0) || (J.thr == 0.0 && S.hros_pos);
    // Available plane (burnable, not harvested, not yet ignited) and Burned plane
    uint32_t *av;
    if constexpr (SMEM) av = s_planes;
    else av = A.avail_scratch + slot * (size_t)A.pw_max;
    uint32_t *brn = A.brn_scratch + slot * (size_t)A.pw_max;
    for (size_t i = tid; i < pw; i += T) { av[i] = __ldg(&J.burnable[i]); brn[i] = 0u; }
    int32_t *istep = J.ign_step ? J.ign_step + (size_t)r * n : nullptr;
    const int32_t sph = J.sph, H = J.hours;
    const int64_t dk = (k & 1) ? J.d_diag : J.d_orth;   // this lane's axis length
    if (tid == 0) {
      S.nnew = 1; S.overflow = 0;
      S.burn[0] = S.burn[1] = 0;
      S.minnext[0] = S.minnext[1] = kNone;
    }
    __syncthreads();

    // Step 1 of Alg. 1: the ignition cell burns from period 0
    int32_t live = 1;
    long long W = 0;          // thread 0's running work count
    int32_t nign = 1;
    {
      const int32_t ic = J.ign_cell[r];
      const int32_t ir = ic / cols, icc = ic - ir * cols;
      if (tid == 0) {
        atomicAnd(&av[(int64_t)ir * wpr + (icc >> 5)], ~(1u << (icc & 31)));
        if (istep) istep[ic] = 0;
      }
      __syncthreads();
      bool open = false;
      if (tid < 8) {
        const int32_t nr = ir + kDR[k], nc = icc + kDC[k];
        open = nr >= 0 && nr < rows && nc >= 0 && nc < cols && plane_bit(av, wpr, nr, nc);
      }
      const uint32_t mask = group_bits(open);   // lanes 0..7 of warp 0 hold the cell's mask
      if (tid < 8) {
        eP[k] = 0;
        ecofs[k] = kNone;
        if (k == 0) { ecell[0] = ic; emask[0] = (uint8_t)mask; enext[0] = kNone; }
      }
      if (tid == 0 && mask == 0) {   // no Available neighbour: Burned after period 1
        atomicOr(&brn[(int64_t)ir * wpr + (icc >> 5)], 1u << (icc & 31));
        S.burn[0] = 1;
      }
      __syncthreads();
      if (S.burn[0]) { live = 0; W = (H * sph >= 1) ? 1 : 0; }
      __syncthreads();
      if (tid == 0) S.burn[0] = 0;
      __syncthreads();
    }
    int32_t cnt = 1;          // entries in the list
    long long s_done = 0;     // last period whose burning count is in W
    int it = 0;               // visited-period counter (parity selects the buffers)
    bool aborted = false;

    for (int32_t h = 0; h < H && live > 0 && !aborted; ++h) {
      const int32_t s0 = h * sph + 1, L = s0 + sph - 1;
      const int64_t *baseh = J.base + (size_t)h * n * 8;
      const int p0 = it & 1;

      // ---- hour boundary (i): drop Burned cells and cells with no open axis
      {
        if (tid == 0) S.out_base = 0;
        __syncthreads();
        for (int32_t b0 = 0; b0 < cnt; b0 += T) {
          const int32_t e = b0 + tid;
          bool keep = false;
          int32_t cell = 0;
          uint32_t mask = 0;
          int64_t P[8];
          if (e < cnt) {
            cell = ecell[e];
            mask = emask[e];
            const int32_t cr = cell / cols, cc = cell - cr * cols;
            keep = mask != 0 && !plane_bit(brn, wpr, cr, cc);
            if (keep) {
#pragma unroll
              for (int q = 0; q < 8; ++q) P[q] = eP[(size_t)e * 8 + q];
            }
          }
          const uint32_t bal = __ballot_sync(0xffffffffu, keep);
          if (lane == 0) S.warp_tot[warp] = __popc(bal);
          __syncthreads();
          int32_t pos = S.out_base + __popc(bal & ((1u << lane) - 1u));
          for (int w = 0; w < warp; ++w) pos += S.warp_tot[w];
          if (keep) {
            ecell[pos] = cell;
            emask[pos] = (uint8_t)mask;
#pragma unroll
            for (int q = 0; q < 8; ++q) eP[(size_t)pos * 8 + q] = P[q];
          }
          __syncthreads();
          if (tid == 0) {
            int32_t tot = 0;
            for (int w = 0; w < T / 32; ++w) tot += S.warp_tot[w];
            S.out_base += tot;
          }
          __syncthreads();
        }
        cnt = S.out_base;
        if (tid == 0) S.nnew = cnt;
      }
      // ---- hour boundary (ii): crossings of this hour, 8 lanes per cell
      for (int32_t e0 = 0; e0 < cnt; e0 += G) {
        const int32_t e = e0 + g;
        const bool act = e < cnt;
        int32_t cell = 0;
        uint32_t mask = 0;
        int64_t P = 0;
        if (act) { cell = ecell[e]; mask = emask[e]; P = eP[(size_t)e * 8 + k]; }
        const int32_t cr = cell / cols, cc = cell - cr * cols;
        bool open = act && ((mask >> k) & 1u);
        if (open) open = plane_bit(av, wpr, cr + kDR[k], cc + kDC[k]);
        mask = group_bits(open);
        uint32_t cof = kNone;
        if (act && (mask != 0 || J.delta > 0.0)) {
          const float f = noise_factor(J.seed, (uint32_t)r, (uint32_t)cell, (uint32_t)h, J.sigma);
          if (open) {
            const int64_t inc = apply_noise(baseh[(size_t)cell * 8 + k], noise_fixed(f), dk);
            const int64_t rem = dk - P;
            if (inc > 0 && inc * sph >= rem) cof = (uint32_t)(ceil_div_small(rem, inc) - 1);
            else P += inc * sph;
          }
          if (J.delta > 0.0 &&
              __dmul_rn(J.hros[(size_t)h * n + cell], (double)f) < J.delta) {   // A5 (i)
            if (k == 0) {
              const uint32_t bit = 1u << (cc & 31);
              if (!(atomicOr(&brn[(int64_t)cr * wpr + (cc >> 5)], bit) & bit))
                atomicAdd(&S.burn[p0], 1);
            }
            if (cof != 0) cof = kNone;   // still sends in period s0, Burned after it
          }
        }
        const uint32_t nx = group_min(cof);
        if (act) {
          ecofs[(size_t)e * 8 + k] = (uint8_t)cof;
          eP[(size_t)e * 8 + k] = P;
          if (k == 0) { emask[e] = (uint8_t)mask; enext[e] = (uint8_t)nx; }
        }
      }
      __syncthreads();

      // ---- periods of this hour at which some axis reaches a centre
      int32_t s = s0;
      for (;;) {
        const int p = it & 1;
        if (tid == 0) { W += (long long)live * (long long)(s - s_done); s_done = s; }
        const uint32_t o = (uint32_t)(s - s0);
        uint32_t lmin = kNone;
        // (A) send and receive: cells with a crossing at offset o
        for (int32_t b0 = 0; b0 < cnt; b0 += T) {
          const int32_t e = b0 + tid;
          const uint32_t nx = (e < cnt) ? (uint32_t)enext[e] : kNone;
          const bool hit = nx == o;
          if (!hit) lmin = min(lmin, nx);
          uint32_t hits = __ballot_sync(0xffffffffu, hit);
          while (hits) {
            int src[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              src[q] = hits ? __ffs(hits) - 1 : -1;
              if (hits) hits &= hits - 1;
            }
            const int my = src[lane >> 3];
            int32_t ent = __shfl_sync(0xffffffffu, e, my < 0 ? 0 : my);
            if (my < 0) ent = -1;
            uint32_t cof = kNone, mask = 0;
            bool crossed = false;
            if (ent >= 0) {
              cof = ecofs[(size_t)ent * 8 + k];
              crossed = cof == o;
              if (crossed) {
                cof = kNone;
                const int32_t cell = ecell[ent];
                const int32_t cr = cell / cols, cc = cell - cr * cols;
                const int32_t nr = cr + kDR[k], nc = cc + kDC[k];
                if (plane_bit(av, wpr, nr, nc)) {                        // Available
                  const int64_t jc = (int64_t)nr * cols + nc;
                  if (gate_free || receive_ok(J, r, jc, h, n)) {          // else consumed
                    const uint32_t bit = 1u << (nc & 31);
                    if (atomicAnd(&av[(int64_t)nr * wpr + (nc >> 5)], ~bit) & bit) {
                      const int32_t idx = atomicAdd(&S.nnew, 1);
                      if (idx < cap) ecell[idx] = (int32_t)jc; else S.overflow = 1;
                      if (istep) istep[jc] = s;
                    }
                  }
                }
              }
            }
            const uint32_t cbits = group_bits(crossed);
            const uint32_t nx2 = group_min(cof);
            if (ent >= 0) {
              if (crossed) ecofs[(size_t)ent * 8 + k] = kNone;
              if (k == 0) {
                mask = emask[ent];
                emask[ent] = (uint8_t)(mask & ~cbits);
                enext[ent] = (uint8_t)nx2;
                lmin = min(lmin, nx2);
              }
            }
          }
        }
        lmin = warp_min(lmin);
        if (lane == 0) atomicMin(&S.minnext[p], lmin);
        __syncthreads();
        if (tid == 0) { S.burn[p ^ 1] = 0; S.minnext[p ^ 1] = kNone; }
        if (S.overflow) { aborted = true; break; }
        // (C) cells ignited in period s: open axes, first crossings, burn-out tests
        const int32_t c1 = S.nnew;
        lmin = kNone;
        for (int32_t e0 = cnt; e0 < c1; e0 += G) {
          const int32_t e = e0 + g;
          const bool act = e < c1;
          const int32_t cell = act ? ecell[e] : 0;
          const int32_t cr = cell / cols, cc = cell - cr * cols;
          const int32_t nr = cr + kDR[k], nc = cc + kDC[k];
          const bool ingrid = act && nr >= 0 && nr < rows && nc >= 0 && nc < cols;
          const int64_t bk = act ? baseh[(size_t)cell * 8 + k] : 0;   // issue the table load early
          const bool open = ingrid && plane_bit(av, wpr, nr, nc);
          const bool ignq = ingrid && !open && (__ldg(&J.burnable[(int64_t)nr * wpr + (nc >> 5)]) >> (nc & 31)) & 1u;
          uint32_t mask = group_bits(open);
          float f = 1.0f;
          bool have_f = false;
          if (act && J.delta > 0.0) {
            f = noise_factor(J.seed, (uint32_t)r, (uint32_t)cell, (uint32_t)h, J.sigma);
            have_f = true;
            if (__dmul_rn(J.hros[(size_t)h * n + cell], (double)f) < J.delta) {   // A5 (i)
              if (k == 0) {
                const uint32_t bit = 1u << (cc & 31);
                if (!(atomicOr(&brn[(int64_t)cr * wpr + (cc >> 5)], bit) & bit))
                  atomicAdd(&S.burn[p], 1);
              }
              mask = 0;
            }
          }
          uint32_t cof = kNone;
          int64_t P = 0;
          if (act && mask != 0 && s < L) {
            if (!have_f) f = noise_factor(J.seed, (uint32_t)r, (uint32_t)cell, (uint32_t)h, J.sigma);
            if ((mask >> k) & 1u) {
              const int32_t nmax = L - s;
              const int64_t inc = apply_noise(bk, noise_fixed(f), dk);
              if (inc > 0 && inc * nmax >= dk) cof = o + (uint32_t)ceil_div_small(dk, inc);
              else P = inc * nmax;
            }
          }
          const uint32_t nx = group_min(cof);
          if (act) {
            ecofs[(size_t)e * 8 + k] = (uint8_t)cof;
            eP[(size_t)e * 8 + k] = P;
            if (k == 0) { emask[e] = (uint8_t)mask; enext[e] = (uint8_t)nx; lmin = min(lmin, nx); }
            // A5 (ii): the neighbour on this axis (if ignited), and lane 0 also this cell
            if (ignq && !has_available_nbr(av, wpr, rows, cols, nr, nc)) {
              const uint32_t bit = 1u << (nc & 31);
              if (!(atomicOr(&brn[(int64_t)nr * wpr + (nc >> 5)], bit) & bit)) atomicAdd(&S.burn[p], 1);
            }
            if (k == 0 && !has_available_nbr(av, wpr, rows, cols, cr, cc)) {
              const uint32_t bit = 1u << (cc & 31);
              if (!(atomicOr(&brn[(int64_t)cr * wpr + (cc >> 5)], bit) & bit)) atomicAdd(&S.burn[p], 1);
            }
          }
        }
        lmin = warp_min(lmin);
        if (lane == 0) atomicMin(&S.minnext[p], lmin);
        __syncthreads();
        const int32_t added = c1 - cnt;
        nign += added;
        live += added - S.burn[p];
        cnt = c1;
        const uint32_t mn = S.minnext[p];
        ++it;
        const int32_t next = (mn == kNone) ? L + 1 : s0 + (int32_t)mn;
        if (next <= s) {   // cannot happen; never visit a period twice
          if (tid == 0) S.overflow = 2;
          aborted = true;
          break;
        }
        if (live == 0) break;
        s = next;
        if (s > L) break;
      }
      if (!aborted && tid == 0) { W += (long long)live * (long long)(L - s_done); s_done = L; }
    }
    __syncthreads();
    {   // scar plane: burnable cells that are no longer Available
      uint32_t *dst = J.ign_plane + (size_t)r * pw;
      for (size_t i = tid; i < pw; i += T) dst[i] = __ldg(&J.burnable[i]) & ~av[i];
    }
    if (tid == 0) {
      J.work[r] = W;
      J.n_ignited[r] = nign;
      J.status[r] = S.overflow;
    }
    __syncthreads();
  }
}

// Variants: CTA size 64 / 128 / 256, planes in global (g) or shared (s) memory.
__global__ void __launch_bounds__(64, 16) k_frontier_g64(FrontierArgs A) { frontier_body<64, false>(A); }
__global__ void __launch_bounds__(128, 8) k_frontier_g128(FrontierArgs A) { frontier_body<128, false>(A); }
__global__ void __launch_bounds__(256, 4) k_frontier_g256(FrontierArgs A) { frontier_body<256, false>(A); }
__global__ void __launch_bounds__(64, 16) k_frontier_s64(FrontierArgs A) { frontier_body<64, true>(A); }
__global__ void __launch_bounds__(128, 8) k_frontier_s128(FrontierArgs A) { frontier_body<128, true>(A); }
__global__ void __launch_bounds__(256, 4) k_frontier_s256(FrontierArgs A) { frontier_body<256, true>(A); }

// ------------------------------------------------------------------ K4
// counts[c] = sum over replicas of the scar bit of c.  Each thread owns one
// 32-cell word and adds the replicas' words into a bit-sliced (vertical)
// counter: plane i holds bit i of the 32 per-cell counts.
__global__ void k_burn_prob(const uint32_t *__restrict__ planes, int32_t R, int32_t rows,
                            int32_t cols, int32_t wpr, int32_t r_chunk, uint32_t *counts,
                            int32_t accumulate) {
  const int64_t pw = (int64_t)rows * wpr;
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= pw) return;
  const int32_t r0 = blockIdx.y * r_chunk;
  const int32_t r1 = min(R, r0 + r_chunk);
  uint32_t c[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) c[i] = 0;
  for (int32_t r = r0; r < r1; ++r) {
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

}  // namespace c2f
