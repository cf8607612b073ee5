// c2f_static.cu -- c2f_frontier_static: the frontier kernel for callers that
// cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc at all: a host
// application that has handed all device memory to its own allocator and
// forbids others to take more, or a plugin loaded into such a host that may
// not allocate after start-up.  For them this entry point runs the frontier
// step (ignited replicas -> scars, work counts) with every byte of scratch
// taken from one file-scope device array of fixed size, kStaticScratchBytes.
// The caller passes the inputs (burnable plane, rate-of-spread table,
// ignition cells) and the outputs in device memory.  No cudaMalloc, cudaFree
// or allocating library routine is called.
//
// The call is synchronous: it copies small arguments into the array, waits
// for the stream, reads the per-replica statuses on the host and re-runs
// replicas whose burning lists overflowed.  It must therefore not be issued
// on a stream that is being captured into a CUDA graph.
//
// Every GPU that loads the library keeps this array until the process exits.
// All calls share it and it keeps the last call's contents; the parts that
// must start at zero are cleared by each call.  Calls that overlap on the GPU
// (on different streams, or from several host threads) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/c2f.h"
#include "c2f_layout.cuh"

namespace c2f {
__global__ void k_frontier_g1(FrontierArgs);
cudaError_t init_device_constants(int device);
}
using namespace c2f;

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;   // 16 MiB
constexpr int32_t kStaticMaxReplicas = 1 << 16;
constexpr int64_t kStaticMinCap = 256;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct DeviceScratch {
  std::once_flag once;
  cudaError_t err = cudaSuccess;
  unsigned char *ptr = nullptr;
};
DeviceScratch g_scratch_of_device[64];

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// carve the array: header (counter, job, item ranges, item list, statuses), then per slot
struct Carve {
  size_t off_counter, off_job, off_begin, off_list, off_status, off_slots;
  size_t per_slot;
  size_t off_cell, off_link, off_cofs, off_P, off_avail, off_brn;   // within the slot area
};

Carve carve(int64_t slots, int64_t cap, int64_t pw, int32_t R) {
  Carve c{};
  size_t o = 0;
  c.off_counter = o; o = align256(o + 8);
  c.off_job = o; o = align256(o + sizeof(SimJob));
  c.off_begin = o; o = align256(o + 2 * sizeof(int64_t));
  c.off_list = o; o = align256(o + sizeof(int64_t) * (size_t)R);
  c.off_status = o; o = align256(o + sizeof(int32_t) * (size_t)R);
  c.off_slots = o;
  // slot-major arrays, each sized for all slots (the kernel indexes slot * cap)
  size_t p = 0;
  c.off_cell = p; p = align256(p + (size_t)slots * cap * 4);
  c.off_link = p; p = align256(p + (size_t)slots * cap * 4);
  c.off_cofs = p; p = align256(p + (size_t)slots * cap * 8);
  c.off_P = p; p = align256(p + (size_t)slots * cap * 64);
  c.off_avail = p; p = align256(p + (size_t)slots * pw * 4);
  c.off_brn = p; p = align256(p + (size_t)slots * pw * 4);
  c.per_slot = p;   // total bytes of the slot area for `slots` slots
  return c;
}

}  // namespace

extern "C" C2F_API int c2f_frontier_static(const c2f_frontier_io *io, const c2f_sim_params *p,
                                           void *stream_ptr) {
  if (!io || !p) return C2F_EINVAL;
  if (io->rows < 1 || io->cols < 1 || io->rows > 65535 || io->cols > 65535) return C2F_EINVAL;
  if (!(io->cell_size_m > 0.0 && io->cell_size_m <= 1e6)) return C2F_EINVAL;
  if (!io->burnable || !io->base || !io->hros || !io->ign_cell || !io->scars || !io->work ||
      !io->n_ignited)
    return C2F_EINVAL;
  if (p->n_replicas < 1 || p->n_replicas > kStaticMaxReplicas) return C2F_EINVAL;
  if (p->hours < 1 || p->minutes_per_step < 1 || 60 % p->minutes_per_step) return C2F_EINVAL;
  if (!(p->ros_sigma >= 0.0 && p->ros_sigma <= 1.0)) return C2F_EINVAL;
  if (!std::isfinite(p->ros_threshold) || !std::isfinite(p->burnout_delta) || p->burnout_delta < 0.0)
    return C2F_EINVAL;
  if (!(p->burn_hours_min == 0 && p->burn_hours_max == 0) &&
      !(p->burn_hours_min >= 1 && p->burn_hours_min <= p->burn_hours_max && p->burn_hours_max <= 24))
    return C2F_EINVAL;
  cudaStream_t st = (cudaStream_t)stream_ptr;
  const int32_t R = p->n_replicas;
  const int32_t wpr = (io->cols + 31) / 32;
  const int64_t pw = (int64_t)io->rows * wpr;
  const int64_t n = (int64_t)io->rows * io->cols;

  // the largest burning list one slot can hold when it has the whole array
  const int64_t header = (int64_t)carve(0, 0, 0, R).off_slots;
  const int64_t avail_bytes = (int64_t)kStaticScratchBytes - header - 8 * 256;
  const int64_t fixed_per_slot = pw * 8;          // Available + Burned planes
  const int64_t per_entry = 4 + 4 + 8 + 64;   // cell, calendar link, crossing offsets, progress
  const int64_t cap_max = std::min<int64_t>(n, (avail_bytes - fixed_per_slot) / per_entry);
  if (cap_max < std::min<int64_t>(n, kStaticMinCap)) return C2F_EINVAL;   // landscape too large

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return C2F_ECUDA; }
  if (init_device_constants(dev) != cudaSuccess) { cudaGetLastError(); return C2F_ECUDA; }   // noise tables
  DeviceScratch &ds = g_scratch_of_device[dev];
  std::call_once(ds.once, [&] {
    void *ptr = nullptr;
    ds.err = cudaGetSymbolAddress(&ptr, g_static_scratch);
    ds.ptr = static_cast<unsigned char *>(ptr);
  });
  if (ds.err != cudaSuccess || !ds.ptr) { cudaGetLastError(); return C2F_ECUDA; }
  unsigned char *base_ptr = ds.ptr;

  SimJob job{};
  job.rows = io->rows; job.cols = io->cols; job.wpr = wpr;
  job.burnable = io->burnable;
  job.base = const_cast<int64_t *>(io->base);
  job.hros = const_cast<double *>(io->hros);
  job.chunk_state = nullptr;   // the caller's table is complete
  job.hour = nullptr;          // receive tests read HROS when the threshold is 0
  job.seed = p->seed;
  job.sigma = (float)p->ros_sigma;
  job.ignition_mode = 0;
  job.thr = p->ros_threshold;
  job.delta = p->burnout_delta;
  job.recv_gate = receive_gate(job.thr, job.const_ros);
  job.sph = 60 / p->minutes_per_step;
  job.hours = p->hours;
  job.burn_min = p->burn_hours_min;   // A5 general condition (1), as in c2f_simulate
  job.burn_max = p->burn_hours_max;
  job.d_orth = (int64_t)std::llrint(io->cell_size_m * 4294967296.0);
  job.d_diag = (int64_t)std::llrint((io->cell_size_m * std::sqrt(2.0)) * 4294967296.0);
  job.n_replicas = R;
  job.ign_plane = io->scars;
  job.ign_step = nullptr;
  job.work = io->work;
  job.n_ignited = io->n_ignited;
  job.ign_cell = const_cast<int32_t *>(io->ign_cell);

  int sm = 0;
  if (cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return C2F_ECUDA;
  }
  std::vector<int64_t> items;   // empty: every replica
  std::vector<int32_t> status(R);
  for (int attempt = 0; attempt < 2; ++attempt) {
    const int64_t todo = items.empty() ? R : (int64_t)items.size();
    int64_t cap, slots;
    if (attempt == 0) {
      cap = std::min<int64_t>(cap_max, std::max<int64_t>(std::min<int64_t>(n, kStaticMinCap),
                                                         std::min<int64_t>(n, 4096)));
      slots = std::max<int64_t>(1, (avail_bytes) / (fixed_per_slot + cap * per_entry));
      slots = std::min<int64_t>({slots, todo, (int64_t)sm * 16});
    } else {
      cap = cap_max;   // one slot with the whole array
      slots = 1;
    }
    // shrink until the carve (with its 256-byte alignment) fits the array
    while (slots > 1 && carve(slots, cap, pw, R).off_slots + carve(slots, cap, pw, R).per_slot > kStaticScratchBytes)
      --slots;
    while (cap > 1 && carve(slots, cap, pw, R).off_slots + carve(slots, cap, pw, R).per_slot > kStaticScratchBytes)
      cap -= std::max<int64_t>(1, cap / 64);
    const Carve c = carve(slots, cap, pw, R);
    if (c.off_slots + c.per_slot > kStaticScratchBytes) return C2F_EINVAL;
    unsigned char *sl = base_ptr + c.off_slots;
    FrontierArgs A{};
    A.jobs = reinterpret_cast<const SimJob *>(base_ptr + c.off_job);
    A.n_jobs = 1;
    A.item_begin = reinterpret_cast<const int64_t *>(base_ptr + c.off_begin);
    A.item_list = items.empty() ? nullptr : reinterpret_cast<const int64_t *>(base_ptr + c.off_list);
    A.n_items = todo;
    A.counter = reinterpret_cast<unsigned long long *>(base_ptr + c.off_counter);
    A.cap = (int32_t)cap;
    A.ent_cell = reinterpret_cast<int32_t *>(sl + c.off_cell);
    A.ent_link = reinterpret_cast<int32_t *>(sl + c.off_link);
    A.ent_cofs = sl + c.off_cofs;
    A.ent_P = reinterpret_cast<int64_t *>(sl + c.off_P);
    A.pw_max = pw;
    A.avail_scratch = reinterpret_cast<uint32_t *>(sl + c.off_avail);
    A.brn_scratch = reinterpret_cast<uint32_t *>(sl + c.off_brn);
    job.status = reinterpret_cast<int32_t *>(base_ptr + c.off_status);
    const int64_t begin[2] = {0, R};
    cudaError_t e = cudaMemcpyAsync(base_ptr + c.off_job, &job, sizeof job, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(base_ptr + c.off_begin, begin, sizeof begin, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !items.empty())
      e = cudaMemcpyAsync(base_ptr + c.off_list, items.data(), sizeof(int64_t) * items.size(),
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base_ptr + c.off_counter, 0, 8, st);
    if (e == cudaSuccess && attempt == 0)
      e = cudaMemsetAsync(base_ptr + c.off_status, 0, sizeof(int32_t) * (size_t)R, st);
    if (e != cudaSuccess) { cudaGetLastError(); return C2F_ECUDA; }
    k_frontier_g1<<<(unsigned)slots, 32, 0, st>>>(A);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(status.data(), base_ptr + c.off_status, sizeof(int32_t) * (size_t)R,
                          cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaGetLastError(); return C2F_ECUDA; }
    items.clear();
    for (int32_t r = 0; r < R; ++r) {
      if (status[r] == 3) return C2F_EINVAL;   // ignition cell outside the grid or not burnable
      if (status[r] > 1) return C2F_ECUDA;
      if (status[r] == 1) items.push_back(r);
    }
    if (items.empty()) return C2F_OK;
    // the re-run starts those replicas from scratch (the kernel clears its planes)
    for (int64_t r : items) {
      if (cudaMemsetAsync(base_ptr + c.off_status + 4 * r, 0, 4, st) != cudaSuccess) {
        cudaGetLastError();
        return C2F_ECUDA;
      }
    }
  }
  return C2F_ENOMEM;   // a burning list outgrew the whole static array
}
