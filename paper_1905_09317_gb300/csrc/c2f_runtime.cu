// c2f_runtime.cu -- host runtime behind the C ABI of include/c2f.h.
//
// Objects and ownership
//   Landscape  device copies of the fuel / slope / aspect grids, the burnable
//              bit plane and list, the cell order and hoisted per-cell FBP
//              terms, the weather stream, and the current rate-of-spread
//              Table (shared_ptr: a simulation keeps the table it ran on alive
//              even if the landscape gets a new one meanwhile).
//   Sim        one simulation: its parameters, its landscape and table, and the
//              per-replica outputs (scar planes, optional ignition steps,
//              counters, status); state PENDING -> RUNNING -> DONE (or
//              CANCELED / FAILED).
//   Epoch      one launch of the frontier kernel over the replicas of one or
//              more simulations, with its own stream, scratch and completion
//              event.  c2f_simulate / c2f_simulate_batch run one epoch to
//              completion; c2f_submit queues simulations and c2f_pump forms
//              epochs from whatever is queued (continuous batching: new
//              requests join the next epoch while earlier epochs still run,
//              and epochs overlap on the device), subject to a free-HBM check.
// Device memory comes from the stream-ordered allocator (cudaMallocAsync) so
// that allocation never synchronises the device.  A replica whose burning
// list outgrows its capacity is re-run with a larger one, so results never
// depend on launch shapes or capacities.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>   // header-only; the ranges cost a pointer test unless a tool is attached

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <list>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/c2f.h"
#include "c2f_layout.cuh"

namespace c2f {
__global__ void k_burnable_plane(const uint8_t *, const uint8_t *, int32_t, int32_t, int32_t,
                                 uint32_t *, int32_t *);
__global__ void k_scan_counts(const int32_t *, int64_t, int32_t *, int32_t *);
__global__ void k_burnable_list(const uint32_t *, const int32_t *, int32_t, int32_t, int32_t,
                                int32_t *);
__global__ void k_cell_prep(const float *, const float *, int64_t, CellPrep *);
__global__ void k_hour_prep(const double *, int32_t, double, HourPrep *);
__global__ void k_ros_table(RosTableArgs);
__global__ void k_order_count(const uint8_t *, const float *, const uint32_t *, int32_t, int32_t,
                              int32_t, int32_t *);
__global__ void k_order_scan(int32_t *);
__global__ void k_order_scatter(const uint8_t *, const float *, const uint32_t *, int32_t, int32_t,
                                int32_t, int32_t *, int32_t *);
__global__ void k_ignite(const SimJob *, int32_t);
__global__ void k_frontier_g1(FrontierArgs);
__global__ void k_frontier_g2(FrontierArgs);
__global__ void k_frontier_g4(FrontierArgs);
__global__ void k_frontier_w1(FrontierArgs);
__global__ void k_frontier_w2(FrontierArgs);
__global__ void k_frontier_w4(FrontierArgs);
__global__ void k_frontier_lg1(FrontierArgs);
__global__ void k_frontier_lw1(FrontierArgs);
__global__ void k_frontier_pg1(FrontierArgs);
__global__ void k_frontier_pw1(FrontierArgs);
__global__ void k_frontier_plg1(FrontierArgs);
__global__ void k_frontier_plw1(FrontierArgs);
__global__ void k_burn_prob(const uint32_t *, int32_t, int32_t, int32_t, int32_t, int32_t,
                            uint32_t *, int32_t, const int32_t *, int32_t);
__global__ void k_scar_bytes(const uint32_t *, int32_t, int32_t, int32_t, int32_t, uint8_t *);
__global__ void k_scar_at_step(const int32_t *, int64_t, int32_t, uint8_t *);
__global__ void k_compare_hours(const int32_t *, const int32_t *, int64_t, int32_t, int32_t, double *, double *,
                                double *);
__global__ void k_compare_final(const uint32_t *, const uint32_t *, int64_t, double *);
__global__ void k_dfma_peak(double *, int32_t);
cudaError_t init_device_constants(int device);
}  // namespace c2f

using namespace c2f;

namespace {

// ------------------------------------------------------------------ device buffers
// A device buffer, stream-ordered: freed on the stream it was allocated on,
// through the context's allocation hooks when it has them.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  const c2f_alloc_hooks *hooks = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { reset(); }
  void reset() {
    if (p) {
      if (hooks) hooks->free(p, bytes, st, hooks->user);
      else cudaFreeAsync(p, st);
    }
    p = nullptr;
    bytes = 0;
  }
  template <class T> T *as() const { return static_cast<T *>(p); }
};

struct TableKey {
  int32_t hours = 0, dt = 0, ellipse = 0;
  double pc = 0, curing = 0, const_ros = 0, const_bros = 0, const_lb = 0;
  bool same_options(const TableKey &o) const {
    return dt == o.dt && ellipse == o.ellipse && pc == o.pc && curing == o.curing &&
           const_ros == o.const_ros && const_bros == o.const_bros && const_lb == o.const_lb;
  }
};

// The rate-of-spread table of a landscape under one set of options.  Eager:
// every row written by K1.  Lazy: rows written on demand by the frontier, 32
// cells at a time, tracked by chunk_state ([hours][rows*wpr], 0 = empty).
struct Table {
  TableKey key;
  // n_scen weather scenarios: n_scen stacked tables of key.hours hours each,
  // hour preps [n_scen][prep_hours]; `weather` holds the scenarios' streams
  // ([n_scen][prep_hours][4] doubles) and then their thresholds (n_scen uint64)
  int32_t n_scen = 1, prep_hours = 0;
  std::shared_ptr<DevBuf> weather;
  DevBuf hour_prep, base, hros, chunk_state;
  bool eager = false;
  bool issued = false;   // its build (K1 or the cleared chunk states) has been issued
  int64_t serial = 0;    // build number within the context (trace tag)
  cudaEvent_t ready = nullptr;   // recorded after the build; epochs on other streams wait on it
  Table() = default;
  Table(const Table &) = delete;
  Table &operator=(const Table &) = delete;
  ~Table() { if (ready) cudaEventDestroy(ready); }
};

struct Landscape {
  int32_t rows = 0, cols = 0, wpr = 0;
  int64_t n = 0;
  double cell_size = 0;
  int32_t n_burnable = 0;
  std::vector<uint8_t> burnable_host;   // validation of fixed ignition cells
  DevBuf fuel, slope, aspect, burnable, burnable_list, cell_prep, order;
  bool has_slope = false;
  int32_t n_hours = 0;
  int32_t n_scen = 1;                   // weather scenarios (Sec. 3.1, uncertainty (3))
  std::vector<double> weather;          // n_scen x n_hours x 4
  std::shared_ptr<DevBuf> weather_dev;  // the same, then n_scen uint64 thresholds
  std::shared_ptr<Table> table;
};

enum SimState { S_PENDING = 0, S_RUNNING, S_DONE, S_CANCELED, S_FAILED };

struct Sim {
  c2f_sim_params p{};
  std::shared_ptr<Landscape> land;
  std::shared_ptr<Table> table;
  int32_t rows = 0, cols = 0, wpr = 0;
  int64_t n = 0;
  DevBuf ign_plane, ign_step, work, n_ignited, ign_cell, status, scen, prof;
  int state = S_PENDING;
  int rc = C2F_OK;
  bool cancel_requested = false;
  int64_t serial = 0;   // creation number within the context (trace tag)
  // asynchronous reads of the buffers on caller streams (burn counts, scar
  // comparison into device memory), one event per stream: the buffers' frees,
  // issued on the streams that allocated them, wait for these reads
  std::vector<std::pair<cudaStream_t, cudaEvent_t>> reads;
  Sim() = default;
  Sim(const Sim &) = delete;
  Sim &operator=(const Sim &) = delete;
  ~Sim() {
    for (auto &r : reads) {
      for (DevBuf *b : {&ign_plane, &ign_step, &work, &n_ignited, &ign_cell, &status, &scen, &prof})
        if (b->p) cudaStreamWaitEvent(b->st, r.second, 0);
      cudaEventDestroy(r.second);   // released once recorded work completes
    }
  }
};

struct Scratch {
  DevBuf ent_cell, ent_link, ent_cofs, ent_P, counter, brn, avail;
  int64_t slots = 0, cap = 0, brn_words = 0, avail_words = 0;
  void reset() {
    ent_cell.reset(); ent_link.reset(); ent_cofs.reset(); ent_P.reset();
    counter.reset(); brn.reset(); avail.reset();
    slots = cap = brn_words = avail_words = 0;
  }
};

struct FrontierPlan {
  std::vector<Landscape *> lands;
  std::vector<Sim *> sims;   // in work-list order
  std::vector<int64_t> begin;
  std::vector<SimJob> jobs;      // host copies stay alive while their uploads are in flight
  std::vector<int64_t> retry;
  DevBuf djobs, dbegin, dlist;
  int64_t cap = 0, max_n = 0, pw_max = 0, n_items = 0;
  bool lazy = false;   // some simulation's table is filled on demand
  void (*kern)(FrontierArgs) = nullptr;
  size_t dyn_smem = 0;
  int threads = 32;
  int64_t ctas = 0;
  FrontierArgs A{};
};

struct Epoch {
  std::vector<std::shared_ptr<Sim>> sims;
  FrontierPlan F;
  Scratch scratch;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};


}  // namespace

struct c2f_ctx {
  int device = 0;
  bool has_hooks = false;
  c2f_alloc_hooks hooks{};
  cudaMemPool_t pool = nullptr;   // the context's stream-ordered pool; keeps freed memory
  int sm_count = 0;
  int smem_optin = 0, smem_per_sm = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  std::recursive_mutex mu;
  std::string last_error;
  int32_t next_id = 1;
  std::unordered_map<int32_t, std::shared_ptr<Landscape>> lands;
  std::unordered_map<int32_t, std::shared_ptr<Sim>> sims;
  // synchronous runs
  Scratch scratch;
  // launch shape
  int frontier_threads = 32;
  bool window_smem = true;
  int warps_per_sm = 0;        // shared-memory sizing target; 0: this launch's own replicas
  bool eager_tables = true;   // simulations build their tables with K1 up front
  int64_t cap_override = 0;
  int compact_eighths = 6;     // compaction trigger within an hour: eighths of the list capacity
  int64_t graph_launches = 0;
  uint32_t wait_limit = 0;     // frontier waits for table chunks: polls before giving up; 0 = default
  // serving
  std::vector<std::shared_ptr<Sim>> pending;
  std::list<std::unique_ptr<Epoch>> inflight;
  std::vector<cudaStream_t> stream_pool;
  int max_inflight = 3;
  int64_t max_epoch_replicas = 1 << 16;
  int64_t hbm_reserve = int64_t(2) << 30;
  int64_t epochs_launched = 0;   // serving statistics
  int64_t admission_waits = 0;   // times queued work was held back for device memory
  cudaStream_t read_stream = nullptr;   // result reads: not queued behind table builds
  cudaStream_t load_stream = nullptr;   // landscape uploads: not queued behind table builds
  // kernel timing
  bool profiling = false;          // kernel-family events (C2F_PROFILE_KERNELS)
  bool replica_counters = false;   // per-replica frontier counters (C2F_PROFILE_REPLICAS)
  // launch trace (c2f_trace): records in caller memory, cursor in the context's
  unsigned long long *trace_rec = nullptr;
  int64_t trace_cap = 0;
  DevBuf trace_cursor;
  int64_t table_serial = 0, sim_serial = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events[C2F_KT_FAMILIES];
  std::vector<cudaEvent_t> event_pool;
};

namespace {

thread_local std::string tl_last_error;   // what c2f_last_error reports to this thread

int fail(c2f_ctx *ctx, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->last_error = buf;
  tl_last_error = buf;
  return code;
}

int cuda_fail(c2f_ctx *ctx, cudaError_t e, const char *what) {
  cudaGetLastError();
  const int code = (e == cudaErrorMemoryAllocation) ? C2F_ENOMEM : C2F_ECUDA;
  return fail(ctx, code, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)

#define CKL(what)                                             \
  do {                                                        \
    cudaError_t e_ = cudaGetLastError();                      \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what);   \
  } while (0)

int dalloc_on(c2f_ctx *ctx, DevBuf &b, size_t bytes, cudaStream_t st) {
  b.reset();
  b.st = st;
  b.hooks = ctx->has_hooks ? &ctx->hooks : nullptr;
  if (bytes == 0) bytes = 16;
  if (b.hooks) {
    b.p = b.hooks->alloc(bytes, st, b.hooks->user);
    if (!b.p) return fail(ctx, C2F_ENOMEM, "allocation hook returned no memory for %zu bytes", bytes);
  } else {
    cudaError_t e = cudaMallocFromPoolAsync(&b.p, bytes, ctx->pool, st);
    if (e != cudaSuccess) {
      b.p = nullptr;
      return cuda_fail(ctx, e, "cudaMallocFromPoolAsync");
    }
  }
  b.bytes = bytes;
  return C2F_OK;
}

int dalloc(c2f_ctx *ctx, DevBuf &b, size_t bytes) { return dalloc_on(ctx, b, bytes, ctx->stream); }

int ensure_device_constants(c2f_ctx *ctx) {
  if (ctx->device < 0 || ctx->device >= 64) return fail(ctx, C2F_EINVAL, "device index out of range");
  const cudaError_t e = init_device_constants(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "uploading constant tables");
  return C2F_OK;
}

cudaEvent_t get_event(c2f_ctx *ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return e;
}

// brackets the launches of one kernel family with events when profiling
// One kernel family's launches: an NVTX range on the host timeline (named for
// the step of the method, for profilers that show or filter by ranges) and,
// with profiling on, a pair of events on the launching stream.
constexpr const char *kFamilyRange[4] = {"c2f K1 rate-of-spread table", "c2f K2 ignition",
                                         "c2f K3 frontier", "c2f K4 burn counts"};
struct ProfScope {
  c2f_ctx *ctx;
  int fam;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  ProfScope(c2f_ctx *c, int f, cudaStream_t s) : ctx(c), fam(f), st(s) {
    nvtxRangePushA(kFamilyRange[f & 3]);
    if (ctx->profiling && (a = get_event(ctx))) cudaEventRecord(a, st);
  }
  ~ProfScope() {
    nvtxRangePop();
    if (!a) return;
    cudaEvent_t b = get_event(ctx);
    if (!b) { ctx->event_pool.push_back(a); return; }
    cudaEventRecord(b, st);
    ctx->prof_events[fam].emplace_back(a, b);
  }
};

unsigned grid1(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

int validate_params(c2f_ctx *ctx, const Landscape &L, const c2f_sim_params *p) {
  if (!p) return fail(ctx, C2F_EINVAL, "params is NULL");
  if (p->n_replicas < 1) return fail(ctx, C2F_EINVAL, "n_replicas must be >= 1");
  if (p->minutes_per_step < 1 || 60 % p->minutes_per_step)
    return fail(ctx, C2F_EINVAL, "minutes_per_step must divide 60");
  if (p->hours < 1) return fail(ctx, C2F_EINVAL, "hours must be >= 1");
  if (p->hours > L.n_hours)
    return fail(ctx, C2F_EINVAL, "hours (%d) exceeds the weather stream (%d hours)", p->hours,
                L.n_hours);
  if (!(p->ros_sigma >= 0.0 && p->ros_sigma <= 1.0))
    return fail(ctx, C2F_EINVAL, "ros_sigma must lie in [0, 1]");
  if (!std::isfinite(p->ros_threshold) || !std::isfinite(p->burnout_delta) ||
      p->burnout_delta < 0.0)
    return fail(ctx, C2F_EINVAL, "threshold / burnout_delta must be finite, delta >= 0");
  if (p->ellipse_mode != 0 && p->ellipse_mode != 1)
    return fail(ctx, C2F_EINVAL, "ellipse_mode must be 0 or 1");
  if (!(p->o1_curing_pct >= 0.0 && p->o1_curing_pct <= 100.0))
    return fail(ctx, C2F_EINVAL, "o1_curing_pct must lie in [0, 100]");
  if (!(p->m1_pc >= 0.0 && p->m1_pc <= 100.0)) return fail(ctx, C2F_EINVAL, "m1_pc must lie in [0, 100]");
  if (!(p->const_ros >= 0.0 && p->const_ros < 1e9)) return fail(ctx, C2F_EINVAL, "const_ros out of range");
  if (!(p->const_bros >= 0.0 && p->const_bros < 1e9) || !(p->const_lb >= 0.0 && p->const_lb <= 1e3))
    return fail(ctx, C2F_EINVAL, "const_bros / const_lb out of range");
  if (!(p->burn_hours_min == 0 && p->burn_hours_max == 0) &&
      !(p->burn_hours_min >= 1 && p->burn_hours_min <= p->burn_hours_max && p->burn_hours_max <= 24))
    return fail(ctx, C2F_EINVAL, "burning hours per day: 0, 0 or 1 <= min <= max <= 24");
  if (p->ignition_mode == 0) {
    if (p->ignition_cell < 0 || p->ignition_cell >= L.n)
      return fail(ctx, C2F_EINVAL, "ignition_cell out of range");
    if (!L.burnable_host[p->ignition_cell])
      return fail(ctx, C2F_EINVAL, "ignition_cell is not burnable");
  } else if (p->ignition_mode == 1) {
    if (L.n_burnable == 0) return fail(ctx, C2F_EINVAL, "landscape has no burnable cell");
  } else {
    return fail(ctx, C2F_EINVAL, "ignition_mode must be 0 or 1");
  }
  return C2F_OK;
}

TableKey key_of(const c2f_sim_params *p) {
  TableKey k;
  k.hours = p->hours;
  k.dt = p->minutes_per_step;
  k.ellipse = p->ellipse_mode;
  k.pc = p->m1_pc;
  k.curing = p->o1_curing_pct;
  k.const_ros = p->const_ros;
  k.const_bros = p->const_ros > 0.0 ? p->const_bros : 0.0;
  k.const_lb = p->const_ros > 0.0 ? p->const_lb : 0.0;
  return k;
}

// a table whose build was never issued (a later step of the call that
// prepared it failed) is not reused: the next call prepares a new one
bool table_ok(const Landscape &L, const TableKey &k) {
  return L.table && L.table->issued && L.table->key.same_options(k) && L.table->key.hours >= k.hours;
}

// A new table object for the options in k (allocation only); the previous one
// stays alive while simulations that ran on it still hold it.  `eager`: the
// table will be filled by K1 (launch_table with eager), so frontiers planned
// before that launch is issued read it as complete (they run after it).
int prepare_table(c2f_ctx *ctx, Landscape &L, const TableKey &k, bool eager) {
  int rc;
  auto T = std::make_shared<Table>();
  T->key = k;
  T->eager = eager;
  T->serial = ++ctx->table_serial;
  T->n_scen = L.n_scen;
  T->prep_hours = L.n_hours;
  T->weather = L.weather_dev;
  const size_t S = (size_t)L.n_scen;
  CK(cudaEventCreateWithFlags(&T->ready, cudaEventDisableTiming));
  if ((rc = dalloc(ctx, T->hour_prep, sizeof(HourPrep) * S * (size_t)L.n_hours))) return rc;
  if ((rc = dalloc(ctx, T->base, sizeof(int64_t) * 8 * S * (size_t)L.n * k.hours))) return rc;
  if ((rc = dalloc(ctx, T->hros, sizeof(double) * S * (size_t)L.n * k.hours))) return rc;
  if ((rc = dalloc(ctx, T->chunk_state, sizeof(uint32_t) * S * (size_t)L.rows * L.wpr * k.hours)))
    return rc;
  L.table = T;
  return C2F_OK;
}

// the context's trace setting as launch arguments (off: rec == nullptr)
TraceArgs trace_args(const c2f_ctx *ctx, int64_t tag) {
  TraceArgs t{};
  if (ctx->trace_rec && ctx->trace_cursor.p) {
    t.rec = ctx->trace_rec;
    t.cursor = ctx->trace_cursor.as<unsigned long long>();
    t.cap = ctx->trace_cap;
    t.tag = tag;
  }
  return t;
}

// K1 over every row of L.table (one launch per weather scenario), then every
// chunk marked done (capturable)
int fill_table(c2f_ctx *ctx, Landscape &L, cudaStream_t st) {
  Table &T = *L.table;
  const TableKey &k = T.key;
  ProfScope prof(ctx, 0, st);
  RosTableArgs a{};
  a.fuel = L.fuel.as<uint8_t>();
  a.slope = L.has_slope ? L.slope.as<float>() : nullptr;
  a.burnable = L.burnable.as<uint32_t>();
  a.rows = L.rows; a.cols = L.cols; a.wpr = L.wpr;
  a.cell = L.cell_prep.as<CellPrep>();
  a.hour = T.hour_prep.as<HourPrep>();
  a.hour0 = 0;
  a.pcf = k.pc / 100.0;
  a.const_ros = k.const_ros;
  a.const_bros = k.const_bros;
  a.const_lb = k.const_lb;
  a.dt2p32 = (double)k.dt * 4294967296.0;
  a.ellipse_mode = k.ellipse;
  a.base = T.base.as<int64_t>();
  a.hros = T.hros.as<double>();
  a.ros8 = nullptr;
  a.order = L.order.as<int32_t>();
  a.trace = trace_args(ctx, T.serial);
  dim3 grid(grid1(L.n, 128), (unsigned)k.hours);
  for (int32_t sc = 0; sc < T.n_scen; ++sc) {
    const size_t rows_off = (size_t)sc * k.hours * (size_t)L.n;
    a.hour = T.hour_prep.as<HourPrep>() + (size_t)sc * T.prep_hours;
    a.base = T.base.as<int64_t>() + rows_off * 8;
    a.hros = T.hros.as<double>() + rows_off;
    k_ros_table<<<grid, 128, 0, st>>>(a);
    CKL("k_ros_table");
  }
  CK(cudaMemsetAsync(T.chunk_state.p, 0x02, T.chunk_state.bytes, st));   // >= 2: done
  T.eager = true;
  return C2F_OK;
}

// a1 (hour prep) for L.table and either K1 (eager) or empty chunk states
// (lazy), on stream st (capturable)
int launch_table(c2f_ctx *ctx, Landscape &L, cudaStream_t st, bool eager) {
  Table &T = *L.table;
  const TableKey &k = T.key;
  {
    ProfScope prof(ctx, 0, st);
    const int32_t nh = T.n_scen * T.prep_hours;   // every scenario's hours, stacked
    k_hour_prep<<<grid1(nh, 64), 64, 0, st>>>(T.weather->as<double>(), nh, k.curing,
                                              T.hour_prep.as<HourPrep>());
    CKL("k_hour_prep");
  }
  if (eager) {
    int rc = fill_table(ctx, L, st);
    if (rc) return rc;
  } else {
    CK(cudaMemsetAsync(T.chunk_state.p, 0, T.chunk_state.bytes, st));
  }
  // inside a graph capture the event is left unrecorded (reads as complete):
  // the graph runs to completion before the capturing call returns
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cs));
  if (cs == cudaStreamCaptureStatusNone) CK(cudaEventRecord(T.ready, st));
  T.issued = true;
  return C2F_OK;
}

// mode 0: an eager table (a lazy one is completed in place); 1: a new eager
// table; 2: a new lazy table
int ensure_table(c2f_ctx *ctx, Landscape &L, const TableKey &k, int mode) {
  if (mode == 0 && table_ok(L, k)) {
    if (L.table->eager) return C2F_OK;
    int rc = fill_table(ctx, L, ctx->stream);
    if (rc) return rc;
    CK(cudaEventRecord(L.table->ready, ctx->stream));
    return C2F_OK;
  }
  int rc = prepare_table(ctx, L, k, mode != 2);
  if (rc) return rc;
  return launch_table(ctx, L, ctx->stream, mode != 2);
}

std::shared_ptr<Landscape> find_land(c2f_ctx *ctx, int32_t id) {
  auto it = ctx->lands.find(id);
  return it == ctx->lands.end() ? nullptr : it->second;
}

std::shared_ptr<Sim> find_sim(c2f_ctx *ctx, int32_t id) {
  auto it = ctx->sims.find(id);
  return it == ctx->sims.end() ? nullptr : it->second;
}

constexpr int64_t kCoRunSmem = 12 * 1024;

int64_t default_cap(const c2f_ctx *ctx, const Landscape &L) {
  if (ctx->cap_override > 0) return std::min<int64_t>(L.n, ctx->cap_override);
  const int64_t c = std::max<int64_t>(1024, 2 * (int64_t)(L.rows + L.cols));
  return std::min<int64_t>(L.n, c);
}

// (a failed allocation releases the whole scratch, so that no buffer is left
// behind sizes that claim it is large enough)
int ensure_scratch(c2f_ctx *ctx, Scratch &S, cudaStream_t st, int64_t slots, int64_t cap, int64_t pw);
int ensure_scratch_once(c2f_ctx *ctx, Scratch &S, cudaStream_t st, int64_t slots, int64_t cap, int64_t pw) {
  int rc;
  if (!(slots <= S.slots && cap <= S.cap && S.ent_cell.p)) {
    slots = std::max(slots, S.slots);
    cap = std::max(cap, S.cap);
    const size_t sc = (size_t)slots * cap;
    if ((rc = dalloc_on(ctx, S.ent_cell, sc * 4, st))) return rc;
    if ((rc = dalloc_on(ctx, S.ent_link, sc * 4, st))) return rc;
    if ((rc = dalloc_on(ctx, S.ent_cofs, sc * 8, st))) return rc;
    if ((rc = dalloc_on(ctx, S.ent_P, sc * 64, st))) return rc;
    S.slots = slots;
    S.cap = cap;
  }
  if (!S.counter.p && (rc = dalloc_on(ctx, S.counter, 64, st))) return rc;
  if (S.slots * pw > S.brn_words) {
    if ((rc = dalloc_on(ctx, S.brn, (size_t)S.slots * pw * 4, st))) return rc;
    S.brn_words = S.slots * pw;
  }
  if (S.slots * pw > S.avail_words) {
    if ((rc = dalloc_on(ctx, S.avail, (size_t)S.slots * pw * 4, st))) return rc;
    S.avail_words = S.slots * pw;
  }
  return C2F_OK;
}

int ensure_scratch(c2f_ctx *ctx, Scratch &S, cudaStream_t st, int64_t slots, int64_t cap, int64_t pw) {
  const int rc = ensure_scratch_once(ctx, S, st, slots, cap, pw);
  if (rc) S.reset();
  return rc;
}

// output buffers of a simulation, allocated and initialised on stream st
int alloc_sim(c2f_ctx *ctx, Sim &s, cudaStream_t st) {
  int rc;
  const Landscape &L = *s.land;
  const int64_t R = s.p.n_replicas;
  const size_t pw = (size_t)L.rows * L.wpr;
  if ((rc = dalloc_on(ctx, s.ign_plane, pw * 4 * R, st))) return rc;
  if (s.p.outputs & C2F_OUT_IGN_STEPS) {
    if ((rc = dalloc_on(ctx, s.ign_step, (size_t)L.n * 4 * R, st))) return rc;
    CK(cudaMemsetAsync(s.ign_step.p, 0xFF, (size_t)L.n * 4 * R, st));
  }
  if ((rc = dalloc_on(ctx, s.work, 8 * R, st))) return rc;
  if ((rc = dalloc_on(ctx, s.n_ignited, 4 * R, st))) return rc;
  if ((rc = dalloc_on(ctx, s.ign_cell, 4 * R, st))) return rc;
  if ((rc = dalloc_on(ctx, s.status, 4 * R, st))) return rc;
  CK(cudaMemsetAsync(s.status.p, 0, 4 * R, st));
  if (s.table->n_scen > 1) {
    if ((rc = dalloc_on(ctx, s.scen, 4 * R, st))) return rc;
  }
  if (ctx->replica_counters) {   // per-replica profile counters of the frontier
    if ((rc = dalloc_on(ctx, s.prof, 8 * kProfCounters * R, st))) return rc;
    CK(cudaMemsetAsync(s.prof.p, 0, 8 * kProfCounters * R, st));
  }
  return C2F_OK;
}

SimJob job_of(const Sim &s) {
  const Landscape &L = *s.land;
  const Table &T = *s.table;
  SimJob j{};
  j.rows = L.rows; j.cols = L.cols; j.wpr = L.wpr;
  j.n_burnable = L.n_burnable;
  j.burnable = L.burnable.as<uint32_t>();
  j.burnable_list = L.burnable_list.as<int32_t>();
  j.base = T.base.as<int64_t>();
  j.hros = T.hros.as<double>();
  j.chunk_state = T.eager ? nullptr : T.chunk_state.as<uint32_t>();
  j.hour = T.hour_prep.as<HourPrep>();
  j.fuel = L.fuel.as<uint8_t>();
  j.slope = L.has_slope ? L.slope.as<float>() : nullptr;
  j.cell = L.cell_prep.as<CellPrep>();
  j.pcf = T.key.pc / 100.0;
  j.const_ros = T.key.const_ros;
  j.const_bros = T.key.const_bros;
  j.const_lb = T.key.const_lb;
  j.dt2p32 = (double)T.key.dt * 4294967296.0;
  j.ellipse_mode = T.key.ellipse;
  j.n_scen = T.n_scen;
  j.scen_hours = T.key.hours;
  j.prep_hours = T.prep_hours;
  j.scen_thr = T.n_scen > 1
      ? reinterpret_cast<const uint64_t *>(T.weather->as<double>() + (size_t)T.n_scen * T.prep_hours * 4)
      : nullptr;
  j.scen = s.scen.as<int32_t>();
  j.seed = s.p.seed;
  j.sigma = (float)s.p.ros_sigma;
  j.ignition_mode = s.p.ignition_mode;
  j.ignition_cell = s.p.ignition_cell;
  j.thr = s.p.ros_threshold;
  j.delta = s.p.burnout_delta;
  j.recv_gate = receive_gate(j.thr, j.const_ros);
  j.sph = 60 / s.p.minutes_per_step;
  j.hours = s.p.hours;
  j.burn_min = s.p.burn_hours_min;
  j.burn_max = s.p.burn_hours_max;
  j.d_orth = (int64_t)std::llrint(L.cell_size * 4294967296.0);
  j.d_diag = (int64_t)std::llrint((L.cell_size * std::sqrt(2.0)) * 4294967296.0);
  j.n_replicas = s.p.n_replicas;
  j.ign_plane = s.ign_plane.as<uint32_t>();
  j.ign_step = s.ign_step.as<int32_t>();
  j.work = s.work.as<int64_t>();
  j.n_ignited = s.n_ignited.as<int32_t>();
  j.ign_cell = s.ign_cell.as<int32_t>();
  j.status = s.status.as<int32_t>();
  j.prof = s.prof.as<long long>();
  j.trace_tag = s.serial;
  return j;
}

// ------------------------------------------------------------------ frontier epochs
// Frontier over the replicas of several simulations: one work list of
// (simulation, replica) items, simulations ordered longest-expected-first so
// that the long replicas start early.  plan_frontier allocates and uploads
// (not capturable), launch_frontier issues K2 and the K3 launch (capturable
// in a CUDA graph), finish_frontier reads the per-replica status and re-runs,
// with a larger burning list, any replica whose list overflowed.
cudaStream_t take_stream(c2f_ctx *ctx);

int64_t replica_cost(const Landscape &L, const Sim &s) {
  return (int64_t)s.p.hours * std::min<int64_t>(L.n_burnable, 50000);
}

// launch shape for `todo` items at burning-list capacity `cap_in`; attempt 0
// sizes the shared-memory list so that the launch is resident at once (capped
// at 8 warps per SM), later attempts give each replica more room
int shape_frontier(c2f_ctx *ctx, FrontierPlan &F, Scratch &S, cudaStream_t st, int64_t todo,
                   int64_t cap_in, int attempt) {
  int rc;
  // 32, 64 or 128: one replica per warp; the profiling kernels (per-replica
  // counters) are one-warp CTAs
  const int threads = (F.lazy || ctx->replica_counters) ? 32 : ctx->frontier_threads;
  const int wpc = threads / 32;
  int64_t cap = (cap_in + 3) & ~int64_t(3);
  int64_t win_cap = cap;
  {
    const int64_t want = std::max<int64_t>(1, (todo + ctx->sm_count - 1) / ctx->sm_count);
    const int64_t warps_per_sm =
        attempt == 0 ? (ctx->warps_per_sm > 0 ? (int64_t)ctx->warps_per_sm : std::min<int64_t>(want, 8))
                     : std::min<int64_t>(want, 2);
    // per CTA: 1 KB reserved by the system and about 1.3 KB of static shared
    // memory per warp; with the default sizing, kCoRunSmem per SM is left for
    // kernels that run beside the frontier (the next step's or request's table
    // build, burn counts), whose CTAs could not be placed on a full SM
    const int64_t reserve = (attempt == 0 && ctx->warps_per_sm == 0) ? kCoRunSmem : 0;
    const int64_t per_warp = ((int64_t)ctx->smem_per_sm - reserve - (1024 * warps_per_sm) / wpc -
                              1300 * warps_per_sm) / warps_per_sm;
    const int64_t room = (per_warp - 2 * (int64_t)kWinRows * kWinWords * 4 - 512) / 14;
    win_cap = std::min<int64_t>(cap, std::max<int64_t>(256, room & ~int64_t(63)));
    if (attempt > 0) win_cap = std::max<int64_t>(256, room & ~int64_t(63));
    win_cap = std::min<int64_t>(win_cap, 65532);   // shared-memory lists link entries with 16 bits
  }
  const int64_t budget = (int64_t)ctx->smem_optin - 2048;
  const int64_t win_words = 2 * (int64_t)kWinRows * kWinWords + win_cap * 7 / 2;
  // shared-memory lists only when they hold at least 40 % of the default
  // capacity: smaller ones overflow on large fires and those replicas run twice
  const bool use_win = ctx->window_smem && win_words * 4 * wpc <= budget &&
                       (attempt == 0 ? (ctx->warps_per_sm > 0 || 5 * win_cap >= 2 * cap) : win_cap >= cap);
  if (use_win) cap = win_cap;
  const int64_t warp_words = use_win ? win_words : 0;
  F.kern = use_win ? (wpc == 1 ? k_frontier_w1 : wpc == 2 ? k_frontier_w2 : k_frontier_w4)
                   : (wpc == 1 ? k_frontier_g1 : wpc == 2 ? k_frontier_g2 : k_frontier_g4);
  if (F.lazy) F.kern = use_win ? k_frontier_lw1 : k_frontier_lg1;
  if (ctx->replica_counters)
    F.kern = F.lazy ? (use_win ? k_frontier_plw1 : k_frontier_plg1) : (use_win ? k_frontier_pw1 : k_frontier_pg1);
  F.dyn_smem = (size_t)warp_words * 4 * wpc;
  F.threads = threads;
  if (F.dyn_smem > 0) {   // only ever raised: plans made earlier may still be launched
    cudaFuncAttributes fa{};
    CK(cudaFuncGetAttributes(&fa, F.kern));
    if ((int)F.dyn_smem > fa.maxDynamicSharedSizeBytes)
      CK(cudaFuncSetAttribute(F.kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F.dyn_smem));
  }
  int bps = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, F.kern, threads, F.dyn_smem));
  bps = std::max(bps, 1);
  const int64_t max_ctas = (int64_t)ctx->sm_count * bps;
  F.ctas = std::min<int64_t>((todo + wpc - 1) / wpc, max_ctas);
  const int64_t slots = F.ctas * wpc;   // one warp per slot
  if ((rc = ensure_scratch(ctx, S, st, slots, cap, F.pw_max))) return rc;
  FrontierArgs &A = F.A;
  A = FrontierArgs{};
  A.jobs = F.djobs.as<SimJob>();
  A.n_jobs = (int32_t)F.sims.size();
  A.item_begin = F.dbegin.as<int64_t>();
  A.item_list = nullptr;
  A.n_items = todo;
  A.counter = S.counter.as<unsigned long long>();
  A.cap = (int32_t)cap;
  A.ent_cell = S.ent_cell.as<int32_t>();
  A.ent_link = S.ent_link.as<int32_t>();
  A.ent_cofs = S.ent_cofs.as<uint8_t>();
  A.ent_P = S.ent_P.as<int64_t>();
  A.pw_max = F.pw_max;
  A.brn_scratch = S.brn.as<uint32_t>();
  A.avail_scratch = S.avail.as<uint32_t>();
  A.smem_warp_words = warp_words;
  A.wait_limit = ctx->wait_limit;
  A.compact_at = (int32_t)std::max<int64_t>(1, std::min<int64_t>(cap - 1, cap * ctx->compact_eighths / 8));
  A.trace = trace_args(ctx, 0);
  F.cap = cap;
  return C2F_OK;
}

int plan_frontier(c2f_ctx *ctx, const std::vector<Sim *> &sims, FrontierPlan &F, Scratch &S,
                  cudaStream_t st) {
  const int32_t nj = (int32_t)sims.size();
  std::vector<int32_t> order(nj);
  for (int32_t i = 0; i < nj; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return replica_cost(*sims[a]->land, *sims[a]) > replica_cost(*sims[b]->land, *sims[b]);
  });
  F.lands.clear();
  F.sims.clear();
  for (int32_t i : order) { F.lands.push_back(sims[i]->land.get()); F.sims.push_back(sims[i]); }
  std::vector<SimJob> &jobs = F.jobs;
  jobs.assign(nj, SimJob{});
  F.begin.assign(nj + 1, 0);
  F.cap = 0; F.max_n = 0; F.pw_max = 0;
  F.lazy = false;
  for (int32_t i = 0; i < nj; ++i) {
    jobs[i] = job_of(*F.sims[i]);
    if (jobs[i].chunk_state) F.lazy = true;
    F.begin[i + 1] = F.begin[i] + F.sims[i]->p.n_replicas;
    F.cap = std::max(F.cap, default_cap(ctx, *F.lands[i]));
    F.max_n = std::max(F.max_n, F.lands[i]->n);
    F.pw_max = std::max<int64_t>(F.pw_max, (int64_t)F.lands[i]->rows * F.lands[i]->wpr);
  }
  F.n_items = F.begin[nj];
  int rc;
  if ((rc = dalloc_on(ctx, F.djobs, sizeof(SimJob) * nj, st))) return rc;
  if ((rc = dalloc_on(ctx, F.dbegin, sizeof(int64_t) * (nj + 1), st))) return rc;
  CK(cudaMemcpyAsync(F.djobs.p, jobs.data(), sizeof(SimJob) * nj, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(F.dbegin.p, F.begin.data(), sizeof(int64_t) * (nj + 1), cudaMemcpyHostToDevice, st));
  return shape_frontier(ctx, F, S, st, F.n_items, F.cap, 0);
}

int launch_frontier(c2f_ctx *ctx, FrontierPlan &F, Scratch &S, cudaStream_t st) {
  {
    ProfScope prof(ctx, 1, st);
    for (size_t i = 0; i < F.sims.size(); ++i) {
      k_ignite<<<grid1(F.sims[i]->p.n_replicas, 128), 128, 0, st>>>(F.djobs.as<SimJob>(), (int32_t)i);
      CKL("k_ignite");
    }
  }
  CK(cudaMemsetAsync(S.counter.p, 0, 8, st));
  ProfScope prof(ctx, 2, st);
  F.kern<<<(unsigned)F.ctas, F.threads, F.dyn_smem, st>>>(F.A);
  CKL("k_frontier");
  return C2F_OK;
}

int finish_frontier(c2f_ctx *ctx, FrontierPlan &F, Scratch &S, cudaStream_t st) {
  int rc;
  const int32_t nj = (int32_t)F.sims.size();
  for (int attempt = 1;; ++attempt) {
    std::vector<int64_t> failed;
    for (int32_t i = 0; i < nj; ++i) {
      const int32_t R = F.sims[i]->p.n_replicas;
      std::vector<int32_t> stv(R);
      CK(cudaMemcpyAsync(stv.data(), F.sims[i]->status.p, 4 * (size_t)R, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int32_t r = 0; r < R; ++r) {
        if (stv[r] == 4)
          return fail(ctx, C2F_ETIMEOUT, "a wait for a table chunk ran out (replica %d)", r);
        if (stv[r] == 3) return fail(ctx, C2F_EINVAL, "ignition cell not burnable (replica %d)", r);
        if (stv[r] > 1) return fail(ctx, C2F_ECUDA, "internal frontier error (replica %d)", r);
        if (stv[r]) failed.push_back(F.begin[i] + r);
      }
    }
    if (failed.empty()) return C2F_OK;
    if (F.cap >= F.max_n) return fail(ctx, C2F_ECUDA, "frontier list overflow at full capacity");
    const int64_t cap = std::min<int64_t>(F.max_n, std::max<int64_t>(F.cap * 4, 1024));
    for (int64_t it : failed) {   // those replicas start again from scratch
      const int32_t i = (int32_t)(std::upper_bound(F.begin.begin(), F.begin.end(), it) - F.begin.begin() - 1);
      const int64_t r = it - F.begin[i];
      Sim &s = *F.sims[i];
      CK(cudaMemsetAsync(s.status.as<int32_t>() + r, 0, 4, st));
      if (s.ign_step.p)
        CK(cudaMemsetAsync(s.ign_step.as<int32_t>() + r * s.n, 0xFF, (size_t)s.n * 4, st));
    }
    if ((rc = shape_frontier(ctx, F, S, st, (int64_t)failed.size(), cap, attempt))) return rc;
    F.retry = failed;
    if ((rc = dalloc_on(ctx, F.dlist, sizeof(int64_t) * F.retry.size(), st))) return rc;
    CK(cudaMemcpyAsync(F.dlist.p, F.retry.data(), sizeof(int64_t) * F.retry.size(), cudaMemcpyHostToDevice, st));
    F.A.item_list = F.dlist.as<int64_t>();
    CK(cudaMemsetAsync(S.counter.p, 0, 8, st));
    {
      ProfScope prof(ctx, 2, st);
      F.kern<<<(unsigned)F.ctas, F.threads, F.dyn_smem, st>>>(F.A);
      CKL("k_frontier(retry)");
    }
    CK(cudaStreamSynchronize(st));
  }
}

// validate + create simulations; their tables are built on ctx->stream (or,
// when `built` is given, allocated and listed for the caller to launch).
// `serving`: tables cover the whole weather stream, so that later requests on
// the landscape reuse them, and output buffers are left for the epoch to
// allocate on its own stream when it is admitted.
int make_sims(c2f_ctx *ctx, int32_t n, const int32_t *ids, const c2f_sim_params *params,
              std::vector<std::shared_ptr<Sim>> &out, std::vector<Landscape *> *built,
              bool serving = false) {
  int rc;
  std::vector<std::shared_ptr<Landscape>> lands(n);
  for (int32_t i = 0; i < n; ++i) {
    lands[i] = find_land(ctx, ids[i]);
    if (!lands[i]) return fail(ctx, C2F_ENOTFOUND, "unknown landscape %d", ids[i]);
    if (lands[i]->n_hours < 1) return fail(ctx, C2F_EINVAL, "landscape %d has no weather", ids[i]);
    if ((rc = validate_params(ctx, *lands[i], &params[i]))) return rc;
  }
  for (int32_t i = 0; i < n; ++i) {
    for (int32_t k = 0; k < i; ++k)
      if (ids[k] == ids[i] && !key_of(&params[k]).same_options(key_of(&params[i])))
        return fail(ctx, C2F_EINVAL, "batch entries %d and %d share a landscape with different ROS options", k, i);
    bool first = true;
    for (int32_t k = 0; k < i; ++k) if (ids[k] == ids[i]) first = false;
    if (!first) continue;
    TableKey want = key_of(&params[i]);
    for (int32_t k = i + 1; k < n; ++k)
      if (ids[k] == ids[i]) want.hours = std::max(want.hours, params[k].hours);
    if (serving && !table_ok(*lands[i], want)) want.hours = std::max(want.hours, lands[i]->n_hours);
    if (!table_ok(*lands[i], want)) {
      if ((rc = prepare_table(ctx, *lands[i], want, ctx->eager_tables))) return rc;
      if (built) built->push_back(lands[i].get());
      else if ((rc = launch_table(ctx, *lands[i], ctx->stream, ctx->eager_tables))) return rc;
    }
  }
  out.resize(n);
  for (int32_t i = 0; i < n; ++i) {
    auto s = std::make_shared<Sim>();
    s->serial = ++ctx->sim_serial;
    s->p = params[i];
    s->land = lands[i];
    s->table = lands[i]->table;
    s->rows = lands[i]->rows; s->cols = lands[i]->cols; s->wpr = lands[i]->wpr; s->n = lands[i]->n;
    out[i] = s;
  }
  return C2F_OK;
}

void register_sims(c2f_ctx *ctx, std::vector<std::shared_ptr<Sim>> &sims, int32_t *ids) {
  for (size_t i = 0; i < sims.size(); ++i) {
    const int32_t id = ctx->next_id++;
    ctx->sims[id] = sims[i];
    ids[i] = id;
  }
}

// synchronous: the simulations of one call, run to completion.
//
// When the call builds tables for several landscapes, the landscapes are cut
// into up to four groups by table cost (largest first, about equal build
// time per group) and each group's frontier is launched on its own stream as
// soon as the group's tables are built, so table builds (FP64-bound) overlap
// the frontiers (latency-bound) of earlier groups.  A batch's launches go out
// as one CUDA graph (fork/join over the group streams); a single simulation
// is launched directly.
int simulate_many(c2f_ctx *ctx, int32_t n, const int32_t *ids, const c2f_sim_params *params,
                  int32_t *sim_ids) {
  if (n < 1 || !ids || !params || !sim_ids) return fail(ctx, C2F_EINVAL, "bad batch arguments");
  CK(cudaSetDevice(ctx->device));
  int rc;
  const bool graph = n > 1 && !ctx->profiling && !ctx->replica_counters;
  std::vector<Landscape *> builds;
  std::vector<std::shared_ptr<Sim>> sims;
  if ((rc = make_sims(ctx, n, ids, params, sims, &builds))) return rc;
  for (auto &s : sims)   // tables built earlier, possibly on another stream
    if (std::find(builds.begin(), builds.end(), s->land.get()) == builds.end())
      CK(cudaStreamWaitEvent(ctx->stream, s->table->ready, 0));
  for (auto &s : sims)
    if ((rc = alloc_sim(ctx, *s, ctx->stream))) return rc;

  // groups of landscapes to build, largest table first
  auto cost = [](const Landscape *L) {
    return (double)L->n * (double)L->table->key.hours * (double)L->table->n_scen;
  };
  std::stable_sort(builds.begin(), builds.end(),
                   [&](const Landscape *a, const Landscape *b) { return cost(a) > cost(b); });
  const int G = (int)std::min<size_t>(4, std::max<size_t>(1, builds.size()));
  std::vector<int> group_of_build(builds.size(), 0);
  {
    double total = 0.0, acc = 0.0;
    for (Landscape *L : builds) total += cost(L);
    for (size_t i = 0; i < builds.size(); ++i) {
      group_of_build[i] = std::min(G - 1, (int)(acc * G / std::max(total, 1.0)));
      acc += cost(builds[i]);
    }
  }
  std::vector<std::vector<Sim *>> gsims(G);
  for (auto &s : sims) {
    int g = 0;   // simulations on landscapes with a table already run in the first group
    for (size_t i = 0; i < builds.size(); ++i)
      if (builds[i] == s->land.get()) g = group_of_build[i];
    gsims[g].push_back(s.get());
  }
  std::vector<FrontierPlan> F(G);
  std::vector<Scratch> extra(G > 1 ? G : 0);
  auto scratch_of = [&](int g) -> Scratch & { return G > 1 ? extra[g] : ctx->scratch; };
  for (int g = 0; g < G; ++g)
    if (!gsims[g].empty() && (rc = plan_frontier(ctx, gsims[g], F[g], scratch_of(g), ctx->stream))) return rc;

  std::vector<cudaStream_t> gst(G, ctx->stream);
  std::vector<cudaEvent_t> ev;   // fork and join events
  auto cleanup = [&]() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (int g = 1; g < G; ++g)
      if (gst[g] != ctx->stream) ctx->stream_pool.push_back(gst[g]);
  };
  for (int g = 1; g < G; ++g) {
    gst[g] = take_stream(ctx);
    if (!gst[g]) { gst[g] = ctx->stream; cleanup(); return fail(ctx, C2F_ECUDA, "cannot create a stream"); }
  }
  auto new_event = [&](cudaEvent_t *e) {
    const cudaError_t r = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
    if (r == cudaSuccess) ev.push_back(*e);
    return r;
  };
  // issue: builds of group g, then (fork) group g's frontier on its stream; join at the end
  auto issue = [&]() -> int {
    int lrc = C2F_OK;
    size_t b = 0;
    std::vector<cudaEvent_t> done;
    for (int g = 0; g < G && !lrc; ++g) {
      for (; b < builds.size() && group_of_build[b] == g && !lrc; ++b)
        lrc = launch_table(ctx, *builds[b], ctx->stream, ctx->eager_tables);
      if (lrc || gsims[g].empty()) continue;
      if (gst[g] != ctx->stream) {
        cudaEvent_t fork;
        cudaError_t e = new_event(&fork);
        if (e == cudaSuccess) e = cudaEventRecord(fork, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(gst[g], fork, 0);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "fork");
      }
      lrc = launch_frontier(ctx, F[g], scratch_of(g), gst[g]);
      if (!lrc && gst[g] != ctx->stream) {
        cudaEvent_t join;
        cudaError_t e = new_event(&join);
        if (e == cudaSuccess) e = cudaEventRecord(join, gst[g]);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "join");
        done.push_back(join);
      }
    }
    for (cudaEvent_t j : done) {
      const cudaError_t e = cudaStreamWaitEvent(ctx->stream, j, 0);
      if (e != cudaSuccess && !lrc) lrc = cuda_fail(ctx, e, "join");
    }
    return lrc;
  };
  if (graph) {
    // the builds captured below run only if the graph is launched
    auto unissue = [&]() { for (Landscape *L : builds) L->table->issued = false; };
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    const int lrc = issue();
    cudaGraph_t gr = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &gr);
    if (lrc) { if (gr) cudaGraphDestroy(gr); unissue(); cleanup(); return lrc; }
    if (ce != cudaSuccess) { unissue(); cleanup(); return cuda_fail(ctx, ce, "cudaStreamEndCapture"); }
    cudaGraphExec_t ge = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ge, gr, 0);
    cudaGraphDestroy(gr);
    if (ie != cudaSuccess) { unissue(); cleanup(); return cuda_fail(ctx, ie, "cudaGraphInstantiate"); }
    const cudaError_t le = cudaGraphLaunch(ge, ctx->stream);
    cudaGraphExecDestroy(ge);
    if (le != cudaSuccess) { unissue(); cleanup(); return cuda_fail(ctx, le, "cudaGraphLaunch"); }
    ++ctx->graph_launches;
  } else {
    if ((rc = issue())) { cudaStreamSynchronize(ctx->stream); cleanup(); return rc; }
  }
  for (int g = 0; g < G && !rc; ++g)
    if (!gsims[g].empty()) rc = finish_frontier(ctx, F[g], scratch_of(g), ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  cleanup();
  if (rc) return rc;
  for (auto &s : sims) s->state = S_DONE;
  register_sims(ctx, sims, sim_ids);
  return C2F_OK;
}

// ------------------------------------------------------------------ serving
cudaStream_t take_stream(c2f_ctx *ctx) {
  if (!ctx->stream_pool.empty()) {
    cudaStream_t s = ctx->stream_pool.back();
    ctx->stream_pool.pop_back();
    return s;
  }
  // epochs run at the highest stream priority: their frontier CTAs are placed
  // before table builds queued at the same time on the context stream
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) { cudaGetLastError(); greatest = 0; }
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, greatest) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return s;
}

// device bytes an epoch needs beyond what its simulations already hold
int64_t epoch_bytes(c2f_ctx *ctx, const std::vector<std::shared_ptr<Sim>> &sims) {
  int64_t R = 0, pw = 0, cap = 0, outputs = 0;
  for (auto &s : sims) {
    const int64_t r = s->p.n_replicas, spw = (int64_t)s->rows * s->wpr;
    R += r;
    pw = std::max<int64_t>(pw, spw);
    cap = std::max(cap, default_cap(ctx, *s->land));
    outputs += r * (spw * 4 + 28);   // scar plane, counters, status, scenario
    if (s->p.outputs & C2F_OUT_IGN_STEPS) outputs += r * s->n * 4;
  }
  const int64_t slots = std::min<int64_t>(R, (int64_t)ctx->sm_count * 8);
  return outputs + slots * (cap * 80 + pw * 8) + 4096;
}

// finish the epochs whose work is done (all of them, when `block`)
int reap(c2f_ctx *ctx, bool block) {
  int first_rc = C2F_OK;
  for (auto it = ctx->inflight.begin(); it != ctx->inflight.end();) {
    Epoch &E = **it;
    if (!block) {
      const cudaError_t q = cudaEventQuery(E.done);
      if (q == cudaErrorNotReady) { ++it; continue; }
      if (q != cudaSuccess) return cuda_fail(ctx, q, "cudaEventQuery");
    }
    const int rc = finish_frontier(ctx, E.F, E.scratch, E.stream);
    for (auto &s : E.sims) {
      if (rc) { s->state = S_FAILED; s->rc = rc; }
      else s->state = s->cancel_requested ? S_CANCELED : S_DONE;
    }
    if (rc && !first_rc) first_rc = rc;
    cudaStreamSynchronize(E.stream);
    cudaEventDestroy(E.done);
    E.F.djobs.reset(); E.F.dbegin.reset(); E.F.dlist.reset();
    E.scratch.reset();
    cudaStreamSynchronize(E.stream);   // the scratch frees above are ordered on it
    ctx->stream_pool.push_back(E.stream);
    it = ctx->inflight.erase(it);
  }
  return first_rc;
}

// launch the queued simulations as one epoch when a slot and memory allow
int launch_pending(c2f_ctx *ctx) {
  if (ctx->pending.empty() || (int)ctx->inflight.size() >= ctx->max_inflight) return C2F_OK;
  std::vector<std::shared_ptr<Sim>> batch;
  int64_t R = 0;
  while (!ctx->pending.empty() &&
         (batch.empty() || R + ctx->pending.front()->p.n_replicas <= ctx->max_epoch_replicas)) {
    R += ctx->pending.front()->p.n_replicas;
    batch.push_back(ctx->pending.front());
    ctx->pending.erase(ctx->pending.begin());
  }
  size_t freeb = 0, totalb = 0;
  CK(cudaMemGetInfo(&freeb, &totalb));
  int64_t avail = (int64_t)freeb;
  if (ctx->pool) {   // blocks the context's pool keeps but does not use count as free
    uint64_t reserved = 0, used = 0;
    CK(cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrReservedMemCurrent, &reserved));
    CK(cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrUsedMemCurrent, &used));
    if (reserved > used) avail += (int64_t)(reserved - used);
  }
  if (avail < epoch_bytes(ctx, batch) + ctx->hbm_reserve && !ctx->inflight.empty()) {
    ctx->pending.insert(ctx->pending.begin(), batch.begin(), batch.end());   // admission: wait for memory
    ++ctx->admission_waits;
    return C2F_OK;
  }
  std::unique_ptr<Epoch> E(new Epoch());
  E->sims = batch;
  E->stream = take_stream(ctx);
  if (!E->stream) return fail(ctx, C2F_ECUDA, "cannot create a stream");
  CK(cudaEventCreateWithFlags(&E->done, cudaEventDisableTiming));
  // the epoch waits for its own tables only, not for other builds queued behind them
  std::vector<Sim *> raw;
  int rc = C2F_OK;
  for (auto &s : batch) {
    raw.push_back(s.get());
    s->state = S_RUNNING;
    if (!rc && cudaStreamWaitEvent(E->stream, s->table->ready, 0) != cudaSuccess)
      rc = cuda_fail(ctx, cudaGetLastError(), "cudaStreamWaitEvent");
    if (!rc) rc = alloc_sim(ctx, *s, E->stream);
  }
  if (!rc) rc = plan_frontier(ctx, raw, E->F, E->scratch, E->stream);
  if (!rc) rc = launch_frontier(ctx, E->F, E->scratch, E->stream);
  if (rc) {
    for (auto &s : batch) { s->state = S_FAILED; s->rc = rc; }
    cudaStreamSynchronize(E->stream);
    cudaEventDestroy(E->done);
    ctx->stream_pool.push_back(E->stream);
    return rc;
  }
  CK(cudaEventRecord(E->done, E->stream));
  ctx->inflight.push_back(std::move(E));
  ++ctx->epochs_launched;
  return C2F_OK;
}

int pump(c2f_ctx *ctx) {
  int rc = reap(ctx, false);
  if (rc) return rc;
  return launch_pending(ctx);
}

int sim_ready(c2f_ctx *ctx, const Sim &s) {
  if (s.state == S_DONE) return C2F_OK;
  if (s.state == S_CANCELED) return fail(ctx, C2F_ECANCELED, "simulation was cancelled");
  if (s.state == S_FAILED) return s.rc ? s.rc : C2F_ECUDA;
  return fail(ctx, C2F_EBUSY, "simulation has not finished");
}

#define LOCK std::lock_guard<std::recursive_mutex> lock_(ctx->mu)

}  // namespace

// ====================================================================== C ABI
extern "C" {

C2F_API void c2f_default_params(c2f_sim_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->n_replicas = 1;
  p->hours = 1;
  p->minutes_per_step = 1;
  p->o1_curing_pct = 60.0;
  p->m1_pc = 50.0;
  p->outputs = C2F_OUT_SCARS | C2F_OUT_COUNTERS;
}

C2F_API int c2f_create(c2f_ctx **out, int device) { return c2f_create_with_hooks(out, device, nullptr); }

C2F_API int c2f_create_with_hooks(c2f_ctx **out, int device, const c2f_alloc_hooks *hooks) {
  if (!out) return C2F_EINVAL;
  *out = nullptr;
  if (hooks && (!hooks->alloc || !hooks->free)) return C2F_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return C2F_EINVAL;
  }
  std::unique_ptr<c2f_ctx> holder(new c2f_ctx());
  c2f_ctx *ctx = holder.get();
  ctx->device = device;
  if (hooks) { ctx->hooks = *hooks; ctx->has_hooks = true; }
  CK(cudaSetDevice(device));
  CK(cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device));
  CK(cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  CK(cudaDeviceGetAttribute(&ctx->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device));
  CK(cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking));
  ctx->stream = ctx->own_stream;
  if (!ctx->has_hooks) {
    // a pool of the context's own that keeps what it frees (tables of tens of
    // GB are freed and allocated again step after step); returned at c2f_destroy
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    CK(cudaMemPoolCreate(&ctx->pool, &props));
    uint64_t keep = UINT64_MAX;
    CK(cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep));
  }
  CK(cudaStreamCreateWithFlags(&ctx->read_stream, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&ctx->load_stream, cudaStreamNonBlocking));
  int rc = ensure_device_constants(ctx);
  if (rc) return rc;
  *out = holder.release();
  return C2F_OK;
}

C2F_API int c2f_set_stream(c2f_ctx *ctx, void *stream) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
  return C2F_OK;
}

C2F_API void c2f_destroy(c2f_ctx *ctx) {
  if (!ctx) return;
  {
    LOCK;
    cudaSetDevice(ctx->device);
    reap(ctx, true);
    cudaStreamSynchronize(ctx->stream);
    ctx->pending.clear();
    ctx->sims.clear();
    ctx->lands.clear();
    ctx->scratch.reset();
    ctx->trace_cursor.reset();
    cudaStreamSynchronize(ctx->stream);
    for (int f = 0; f < C2F_KT_FAMILIES; ++f)
      for (auto &pr : ctx->prof_events[f]) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    for (cudaStream_t s : ctx->stream_pool) cudaStreamDestroy(s);
    cudaDeviceSynchronize();
    if (ctx->read_stream) cudaStreamDestroy(ctx->read_stream);
    if (ctx->load_stream) cudaStreamDestroy(ctx->load_stream);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  }
  delete ctx;
}

C2F_API const char *c2f_last_error(const c2f_ctx *ctx) {
  (void)ctx;
  return tl_last_error.c_str();
}

C2F_API int c2f_load_landscape(c2f_ctx *ctx, int32_t rows, int32_t cols, double cell_size_m,
                               const uint8_t *fuel, const float *slope_pct,
                               const float *aspect_deg, const uint8_t *unburnable,
                               int32_t *landscape_id) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  if (!fuel || !landscape_id) return fail(ctx, C2F_EINVAL, "fuel and landscape_id are required");
  if (rows < 1 || cols < 1 || rows > 65535 || cols > 65535 || (int64_t)rows * cols >= (1LL << 31))
    return fail(ctx, C2F_EINVAL, "rows and cols must lie in [1, 65535] and rows*cols < 2^31");
  if (!(cell_size_m > 0.0 && cell_size_m <= 1e6)) return fail(ctx, C2F_EINVAL, "cell_size_m out of range");
  const int64_t n = (int64_t)rows * cols;
  auto L = std::make_shared<Landscape>();
  L->burnable_host.resize(n);
  for (int64_t i = 0; i < n; ++i) {   // one pass: checks and the host copy of the burnable mask
    if (fuel[i] >= F_NCODES)
      return fail(ctx, C2F_EINVAL, "fuel code %d at cell %lld is not in the table", (int)fuel[i], (long long)i);
    if (slope_pct && !(slope_pct[i] >= 0.0f && slope_pct[i] < 1e6f))
      return fail(ctx, C2F_EINVAL, "slope at cell %lld is not a finite value >= 0", (long long)i);
    if (aspect_deg && (!std::isfinite(aspect_deg[i]) || std::fabs(aspect_deg[i]) > 1e6f))
      return fail(ctx, C2F_EINVAL, "aspect at cell %lld is not finite", (long long)i);
    L->burnable_host[i] = (fuel[i] != 0 && !(unburnable && unburnable[i])) ? 1 : 0;
  }
  CK(cudaSetDevice(ctx->device));
  // uploads and set-up kernels on the context's load stream: the waits below
  // are for this landscape's work only, not for table builds queued before it
  cudaStream_t st = ctx->load_stream;
  L->rows = rows; L->cols = cols; L->n = n; L->cell_size = cell_size_m;
  L->wpr = (cols + 31) / 32;
  int rc;
  if ((rc = dalloc_on(ctx, L->fuel, n, st))) return rc;
  CK(cudaMemcpyAsync(L->fuel.p, fuel, n, cudaMemcpyHostToDevice, st));
  L->has_slope = slope_pct != nullptr;
  if (slope_pct) {
    if ((rc = dalloc_on(ctx, L->slope, n * 4, st))) return rc;
    CK(cudaMemcpyAsync(L->slope.p, slope_pct, n * 4, cudaMemcpyHostToDevice, st));
  }
  if (aspect_deg) {
    if ((rc = dalloc_on(ctx, L->aspect, n * 4, st))) return rc;
    CK(cudaMemcpyAsync(L->aspect.p, aspect_deg, n * 4, cudaMemcpyHostToDevice, st));
  }
  DevBuf unb;
  if (unburnable) {
    if ((rc = dalloc_on(ctx, unb, n, st))) return rc;
    CK(cudaMemcpyAsync(unb.p, unburnable, n, cudaMemcpyHostToDevice, st));
  }
  const int64_t words = (int64_t)rows * L->wpr;
  DevBuf wcount, woffs, total;
  if ((rc = dalloc_on(ctx, L->burnable, words * 4, st))) return rc;
  if ((rc = dalloc_on(ctx, wcount, words * 4, st))) return rc;
  if ((rc = dalloc_on(ctx, woffs, words * 4, st))) return rc;
  if ((rc = dalloc_on(ctx, total, 4, st))) return rc;
  k_burnable_plane<<<grid1(words, 256), 256, 0, st>>>(
      L->fuel.as<uint8_t>(), unb.as<uint8_t>(), rows, cols, L->wpr, L->burnable.as<uint32_t>(),
      wcount.as<int32_t>());
  CKL("k_burnable_plane");
  k_scan_counts<<<1, 1024, 0, st>>>(wcount.as<int32_t>(), words, woffs.as<int32_t>(),
                                              total.as<int32_t>());
  CKL("k_scan_counts");
  int32_t nb = 0;
  CK(cudaMemcpyAsync(&nb, total.p, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  L->n_burnable = nb;
  if ((rc = dalloc_on(ctx, L->burnable_list, (size_t)std::max(nb, 1) * 4, st))) return rc;
  k_burnable_list<<<grid1(words, 256), 256, 0, st>>>(
      L->burnable.as<uint32_t>(), woffs.as<int32_t>(), rows, cols, L->wpr,
      L->burnable_list.as<int32_t>());
  CKL("k_burnable_list");
  {   // cells grouped by (fuel, sloped) for the ROS-table kernel
    DevBuf cursor;
    if ((rc = dalloc_on(ctx, L->order, (size_t)n * 4, st))) return rc;
    if ((rc = dalloc_on(ctx, cursor, kOrderBuckets * 4, st))) return rc;
    CK(cudaMemsetAsync(cursor.p, 0, kOrderBuckets * 4, st));
    k_order_count<<<grid1(n, 256), 256, 0, st>>>(L->fuel.as<uint8_t>(), L->slope.as<float>(),
        L->burnable.as<uint32_t>(), rows, cols, L->wpr, cursor.as<int32_t>());
    CKL("k_order_count");
    k_order_scan<<<1, 32, 0, st>>>(cursor.as<int32_t>());
    CKL("k_order_scan");
    k_order_scatter<<<grid1(n, 256), 256, 0, st>>>(L->fuel.as<uint8_t>(), L->slope.as<float>(),
        L->burnable.as<uint32_t>(), rows, cols, L->wpr, cursor.as<int32_t>(), L->order.as<int32_t>());
    CKL("k_order_scatter");
    CK(cudaStreamSynchronize(st));
  }
  if ((rc = dalloc_on(ctx, L->cell_prep, sizeof(CellPrep) * n, st))) return rc;
  k_cell_prep<<<grid1(n, 256), 256, 0, st>>>(L->slope.as<float>(), L->aspect.as<float>(), n,
                                                     L->cell_prep.as<CellPrep>());
  CKL("k_cell_prep");
  CK(cudaStreamSynchronize(st));
  const int32_t id = ctx->next_id++;
  ctx->lands[id] = L;
  *landscape_id = id;
  return C2F_OK;
}

namespace {

// Scenario thresholds (Sec. 3.1, uncertainty (3)): T_s = floor(2^32 cum_s /
// total) with left-to-right binary64 sums, T_{S-1} = 2^32; a replica whose
// Philox word x0 is below T_s and not below T_{s-1} runs scenario s.
bool scenario_thresholds(int32_t n, const double *prob, std::vector<uint64_t> &thr) {
  double total = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    if (!(prob[i] >= 0.0) || !std::isfinite(prob[i])) return false;
    total += prob[i];
  }
  if (!(total > 0.0) || !std::isfinite(total)) return false;
  thr.assign(n, 0);
  double cum = 0.0;
  for (int32_t i = 0; i < n; ++i) {
    cum += prob[i];
    const double q = cum / total;   // <= 1: the partial sums never pass the total
    thr[i] = (i == n - 1) ? (uint64_t(1) << 32) : (uint64_t)(q * 4294967296.0);
  }
  return true;
}

int set_weather_impl(c2f_ctx *ctx, int32_t landscape_id, int32_t n_scen, int32_t n_hours,
                     const c2f_weather_hour *w, const double *prob) {
  auto L = find_land(ctx, landscape_id);
  if (!L) return fail(ctx, C2F_ENOTFOUND, "unknown landscape %d", landscape_id);
  if (n_scen < 1 || n_scen > 4096) return fail(ctx, C2F_EINVAL, "n_scenarios must lie in [1, 4096]");
  if (n_hours < 1 || n_hours > 65535 || !w) return fail(ctx, C2F_EINVAL, "n_hours must lie in [1, 65535]");
  if ((int64_t)n_scen * n_hours > 65535)
    return fail(ctx, C2F_EINVAL, "n_scenarios * n_hours must not exceed 65535");
  std::vector<uint64_t> thr(1, uint64_t(1) << 32);
  if (n_scen > 1 && (!prob || !scenario_thresholds(n_scen, prob, thr)))
    return fail(ctx, C2F_EINVAL, "scenario probabilities must be finite, >= 0 and not all 0");
  const int64_t nh = (int64_t)n_scen * n_hours;
  for (int64_t h = 0; h < nh; ++h) {
    const c2f_weather_hour &x = w[h];
    if (!std::isfinite(x.ws_kmh) || x.ws_kmh < 0 || x.ws_kmh > 1000 || !std::isfinite(x.wd_from_deg) ||
        std::fabs(x.wd_from_deg) > 1e6 || !(x.ffmc >= 0.0 && x.ffmc < 101.0) ||
        !(x.bui > 0.0 && x.bui < 1e6))
      return fail(ctx, C2F_EINVAL, "weather hour %lld out of range", (long long)h);
  }
  CK(cudaSetDevice(ctx->device));
  std::vector<double> host((size_t)nh * 4 + (size_t)n_scen);
  for (int64_t h = 0; h < nh; ++h) {
    host[h * 4 + 0] = w[h].ws_kmh;
    host[h * 4 + 1] = w[h].wd_from_deg;
    host[h * 4 + 2] = w[h].ffmc;
    host[h * 4 + 3] = w[h].bui;
  }
  std::memcpy(host.data() + nh * 4, thr.data(), sizeof(uint64_t) * n_scen);
  // a fresh device copy: tables still being built from the old one keep it
  auto wd = std::make_shared<DevBuf>();
  int rc;
  if ((rc = dalloc(ctx, *wd, sizeof(double) * host.size()))) return rc;
  CK(cudaMemcpyAsync(wd->p, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice,
                     ctx->stream));
  L->n_hours = n_hours;
  L->n_scen = n_scen;
  L->weather = std::move(host);   // the same buffer: the copy's source stays alive
  L->weather.resize((size_t)nh * 4);
  L->weather_dev = wd;
  L->table.reset();   // running simulations keep the table they started with
  return C2F_OK;
}

}  // namespace

C2F_API int c2f_set_weather(c2f_ctx *ctx, int32_t landscape_id, int32_t n_hours,
                            const c2f_weather_hour *w) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  return set_weather_impl(ctx, landscape_id, 1, n_hours, w, nullptr);
}

C2F_API int c2f_set_weather_scenarios(c2f_ctx *ctx, int32_t landscape_id, int32_t n_scenarios,
                                      int32_t n_hours, const c2f_weather_hour *w,
                                      const double *prob) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  return set_weather_impl(ctx, landscape_id, n_scenarios, n_hours, w, prob);
}

C2F_API int c2f_build_ros(c2f_ctx *ctx, int32_t landscape_id, const c2f_sim_params *p, int force) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  if (force < 0 || force > 2) return fail(ctx, C2F_EINVAL, "force must be 0, 1 or 2");
  auto L = find_land(ctx, landscape_id);
  if (!L) return fail(ctx, C2F_ENOTFOUND, "unknown landscape %d", landscape_id);
  if (L->n_hours < 1) return fail(ctx, C2F_EINVAL, "landscape has no weather");
  int rc = validate_params(ctx, *L, p);
  if (rc) return rc;
  CK(cudaSetDevice(ctx->device));
  return ensure_table(ctx, *L, key_of(p), force);
}

C2F_API int c2f_get_ros_scenario(c2f_ctx *ctx, int32_t landscape_id, const c2f_sim_params *p,
                                 int32_t scenario, int32_t hour, double *ros8, double *hros,
                                 int64_t *base) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto L = find_land(ctx, landscape_id);
  if (!L) return fail(ctx, C2F_ENOTFOUND, "unknown landscape %d", landscape_id);
  if (L->n_hours < 1) return fail(ctx, C2F_EINVAL, "landscape has no weather");
  int rc = validate_params(ctx, *L, p);
  if (rc) return rc;
  if (hour < 0 || hour >= p->hours) return fail(ctx, C2F_EINVAL, "hour out of range");
  if (scenario < 0 || scenario >= L->n_scen) return fail(ctx, C2F_EINVAL, "scenario out of range");
  CK(cudaSetDevice(ctx->device));
  if ((rc = ensure_table(ctx, *L, key_of(p), 0))) return rc;
  const Table &T = *L->table;
  CK(cudaStreamWaitEvent(ctx->stream, T.ready, 0));
  const size_t n = (size_t)L->n;
  const size_t row0 = ((size_t)scenario * T.key.hours + hour) * n;   // first row of (scenario, hour)
  if (base)
    CK(cudaMemcpyAsync(base, T.base.as<int64_t>() + row0 * 8, n * 64, cudaMemcpyDeviceToHost,
                       ctx->stream));
  if (hros)
    CK(cudaMemcpyAsync(hros, T.hros.as<double>() + row0, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
  if (ros8) {
    DevBuf tmp;
    if ((rc = dalloc(ctx, tmp, n * 64))) return rc;
    RosTableArgs a{};
    a.fuel = L->fuel.as<uint8_t>();
    a.slope = L->has_slope ? L->slope.as<float>() : nullptr;
    a.burnable = L->burnable.as<uint32_t>();
    a.rows = L->rows; a.cols = L->cols; a.wpr = L->wpr;
    a.cell = L->cell_prep.as<CellPrep>();
    a.hour = T.hour_prep.as<HourPrep>() + (size_t)scenario * T.prep_hours;
    a.hour0 = hour;
    a.pcf = p->m1_pc / 100.0;
    a.const_ros = p->const_ros;
    a.const_bros = p->const_ros > 0.0 ? p->const_bros : 0.0;
    a.const_lb = p->const_ros > 0.0 ? p->const_lb : 0.0;
    a.dt2p32 = (double)p->minutes_per_step * 4294967296.0;
    a.ellipse_mode = p->ellipse_mode;
    a.ros8 = tmp.as<double>();
    k_ros_table<<<dim3(grid1(n, 128), 1), 128, 0, ctx->stream>>>(a);
    CKL("k_ros_table(export)");
    CK(cudaMemcpyAsync(ros8, tmp.p, n * 64, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return C2F_OK;
}

C2F_API int c2f_get_ros(c2f_ctx *ctx, int32_t landscape_id, const c2f_sim_params *p, int32_t hour,
                        double *ros8, double *hros, int64_t *base) {
  return c2f_get_ros_scenario(ctx, landscape_id, p, 0, hour, ros8, hros, base);
}

C2F_API int c2f_simulate(c2f_ctx *ctx, int32_t landscape_id, const c2f_sim_params *p,
                         int32_t *sim_id) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  return simulate_many(ctx, 1, &landscape_id, p, sim_id);
}

C2F_API int c2f_simulate_batch(c2f_ctx *ctx, int32_t n, const int32_t *landscape_ids,
                               const c2f_sim_params *params, int32_t *sim_ids) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  return simulate_many(ctx, n, landscape_ids, params, sim_ids);
}

C2F_API int c2f_submit(c2f_ctx *ctx, int32_t landscape_id, const c2f_sim_params *p, int32_t *sim_id) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  if (!sim_id) return fail(ctx, C2F_EINVAL, "sim_id is NULL");
  CK(cudaSetDevice(ctx->device));
  std::vector<std::shared_ptr<Sim>> sims;
  int rc = make_sims(ctx, 1, &landscape_id, p, sims, nullptr, true);
  if (rc) return rc;
  ctx->pending.push_back(sims[0]);
  register_sims(ctx, sims, sim_id);
  return pump(ctx);
}

C2F_API int c2f_pump(c2f_ctx *ctx) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  CK(cudaSetDevice(ctx->device));
  return pump(ctx);
}

C2F_API int c2f_poll(c2f_ctx *ctx, int32_t sim_id, int32_t *done) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto s = find_sim(ctx, sim_id);
  if (!s) return fail(ctx, C2F_ENOTFOUND, "unknown simulation %d", sim_id);
  CK(cudaSetDevice(ctx->device));
  int rc = pump(ctx);
  if (done) *done = (s->state == S_DONE || s->state == S_CANCELED || s->state == S_FAILED) ? 1 : 0;
  if (s->state == S_FAILED) return s->rc;
  return rc;
}

C2F_API int c2f_wait(c2f_ctx *ctx, int32_t sim_id) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto s = find_sim(ctx, sim_id);
  if (!s) return fail(ctx, C2F_ENOTFOUND, "unknown simulation %d", sim_id);
  CK(cudaSetDevice(ctx->device));
  while (s->state == S_PENDING || s->state == S_RUNNING) {
    int rc = pump(ctx);
    if (rc && s->state != S_FAILED) return rc;
    if (s->state == S_PENDING && ctx->inflight.empty()) return fail(ctx, C2F_ECUDA, "scheduler stalled");
    if ((s->state == S_PENDING || s->state == S_RUNNING) && !ctx->inflight.empty())
      CK(cudaEventSynchronize(ctx->inflight.front()->done));   // the oldest epoch frees a slot
  }
  if (s->state == S_CANCELED) return fail(ctx, C2F_ECANCELED, "simulation was cancelled");
  if (s->state == S_FAILED) return s->rc;
  return C2F_OK;
}

C2F_API int c2f_cancel(c2f_ctx *ctx, int32_t sim_id) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto s = find_sim(ctx, sim_id);
  if (!s) return fail(ctx, C2F_ENOTFOUND, "unknown simulation %d", sim_id);
  if (s->state == S_PENDING) {
    auto it = std::find(ctx->pending.begin(), ctx->pending.end(), s);
    if (it != ctx->pending.end()) ctx->pending.erase(it);
    s->state = S_CANCELED;
  } else if (s->state == S_RUNNING) {
    s->cancel_requested = true;   // its epoch runs to the end; the result is discarded
  }
  return C2F_OK;
}

// counts over all replicas, or (scen) over those that drew weather scenario `want`
// an asynchronous read of s's buffers issued on stream st
static int note_read(c2f_ctx *ctx, Sim &s, cudaStream_t st) {
  for (auto &r : s.reads)
    if (r.first == st) {
      CK(cudaEventRecord(r.second, st));
      return C2F_OK;
    }
  cudaEvent_t e = nullptr;
  CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  s.reads.emplace_back(st, e);
  CK(cudaEventRecord(e, st));
  return C2F_OK;
}

static int burn_prob_into(c2f_ctx *ctx, Sim &s, uint32_t *dst, cudaStream_t st,
                          const int32_t *scen = nullptr, int32_t want = 0) {
  const int32_t R = s.p.n_replicas;
  const int64_t words = (int64_t)s.rows * s.wpr;
  const int64_t target = (int64_t)ctx->sm_count * 4 * 256;
  int32_t chunks = (int32_t)std::min<int64_t>(R, std::max<int64_t>(1, target / std::max<int64_t>(words, 1)));
  int32_t per = (R + chunks - 1) / chunks;
  if (per > 65535) per = 65535;
  chunks = (R + per - 1) / per;
  ProfScope prof(ctx, 3, st);
  if (chunks > 1) CK(cudaMemsetAsync(dst, 0, (size_t)s.n * 4, st));
  k_burn_prob<<<dim3(grid1(words, 256), (unsigned)chunks), 256, 0, st>>>(
      s.ign_plane.as<uint32_t>(), R, s.rows, s.cols, s.wpr, per, dst, chunks > 1 ? 1 : 0, scen, want);
  CKL("k_burn_prob");
  return C2F_OK;
}

C2F_API int c2f_burn_prob(c2f_ctx *ctx, int32_t sim_id, uint32_t *counts) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto s = find_sim(ctx, sim_id);
  if (!s) return fail(ctx, C2F_ENOTFOUND, "unknown simulation %d", sim_id);
  if (!counts) return fail(ctx, C2F_EINVAL, "counts is NULL");
  int rc = sim_ready(ctx, *s);
  if (rc) return rc;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->read_stream;
  DevBuf tmp;
  if ((rc = dalloc_on(ctx, tmp, (size_t)s->n * 4, st))) return rc;
  if ((rc = burn_prob_into(ctx, *s, tmp.as<uint32_t>(), st))) return rc;
  CK(cudaMemcpyAsync(counts, tmp.p, (size_t)s->n * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return C2F_OK;
}

C2F_API int c2f_burn_prob_scenario(c2f_ctx *ctx, int32_t sim_id, int32_t scenario, uint32_t *counts) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto s = find_sim(ctx, sim_id);
  if (!s) return fail(ctx, C2F_ENOTFOUND, "unknown simulation %d", sim_id);
  if (!counts) return fail(ctx, C2F_EINVAL, "counts is NULL");
  int rc = sim_ready(ctx, *s);
  if (rc) return rc;
  if (scenario < 0 || scenario >= s->table->n_scen) return fail(ctx, C2F_EINVAL, "scenario out of range");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->read_stream;
  DevBuf tmp;
  if ((rc = dalloc_on(ctx, tmp, (size_t)s->n * 4, st))) return rc;
  if ((rc = burn_prob_into(ctx, *s, tmp.as<uint32_t>(), st, s->scen.as<int32_t>(), scenario))) return rc;
  CK(cudaMemcpyAsync(counts, tmp.p, (size_t)s->n * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return C2F_OK;
}

C2F_API int c2f_burn_prob_device(c2f_ctx *ctx, int32_t sim_id, uint32_t *counts_dev) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto s = find_sim(ctx, sim_id);
  if (!s) return fail(ctx, C2F_ENOTFOUND, "unknown simulation %d", sim_id);
  if (!counts_dev) return fail(ctx, C2F_EINVAL, "counts_dev is NULL");
  int rc = sim_ready(ctx, *s);
  if (rc) return rc;
  CK(cudaSetDevice(ctx->device));
  if ((rc = burn_prob_into(ctx, *s, counts_dev, ctx->stream))) return rc;
  return note_read(ctx, *s, ctx->stream);
}

C2F_API int c2f_get_scars(c2f_ctx *ctx, int32_t sim_id, uint8_t *scars, int32_t *ign_step) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto s = find_sim(ctx, sim_id);
  if (!s) return fail(ctx, C2F_ENOTFOUND, "unknown simulation %d", sim_id);
  int rc = sim_ready(ctx, *s);
  if (rc) return rc;
  if (ign_step && !s->ign_step.p)
    return fail(ctx, C2F_EINVAL, "simulation did not keep ignition steps (C2F_OUT_IGN_STEPS)");
  CK(cudaSetDevice(ctx->device));
  const int32_t R = s->p.n_replicas;
  const size_t total = (size_t)s->n * R;
  cudaStream_t st = ctx->read_stream;
  if (scars) {
    DevBuf tmp;
    if ((rc = dalloc_on(ctx, tmp, total, st))) return rc;
    k_scar_bytes<<<grid1((int64_t)total, 256), 256, 0, st>>>(
        s->ign_plane.as<uint32_t>(), R, s->rows, s->cols, s->wpr, tmp.as<uint8_t>());
    CKL("k_scar_bytes");
    CK(cudaMemcpyAsync(scars, tmp.p, total, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  if (ign_step) CK(cudaMemcpyAsync(ign_step, s->ign_step.p, total * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return C2F_OK;
}

C2F_API int c2f_get_replica_scar(c2f_ctx *ctx, int32_t sim_id, int32_t replica, uint8_t *scar,
                                 int32_t *ign_step) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto s = find_sim(ctx, sim_id);
  if (!s) return fail(ctx, C2F_ENOTFOUND, "unknown simulation %d", sim_id);
  if (!scar) return fail(ctx, C2F_EINVAL, "scar is NULL");
  int rc = sim_ready(ctx, *s);
  if (rc) return rc;
  if (replica < 0 || replica >= s->p.n_replicas) return fail(ctx, C2F_EINVAL, "replica out of range");
  if (ign_step && !s->ign_step.p)
    return fail(ctx, C2F_EINVAL, "simulation did not keep ignition steps (C2F_OUT_IGN_STEPS)");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->read_stream;
  const size_t pw = (size_t)s->rows * s->wpr;
  DevBuf tmp;
  if ((rc = dalloc_on(ctx, tmp, (size_t)s->n, st))) return rc;
  k_scar_bytes<<<grid1(s->n, 256), 256, 0, st>>>(s->ign_plane.as<uint32_t>() + (size_t)replica * pw, 1,
                                                 s->rows, s->cols, s->wpr, tmp.as<uint8_t>());
  CKL("k_scar_bytes");
  CK(cudaMemcpyAsync(scar, tmp.p, (size_t)s->n, cudaMemcpyDeviceToHost, st));
  if (ign_step)
    CK(cudaMemcpyAsync(ign_step, s->ign_step.as<int32_t>() + (size_t)replica * s->n, (size_t)s->n * 4,
                       cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return C2F_OK;
}

C2F_API int c2f_get_scar_bits(c2f_ctx *ctx, int32_t sim_id, uint32_t *words) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto s = find_sim(ctx, sim_id);
  if (!s) return fail(ctx, C2F_ENOTFOUND, "unknown simulation %d", sim_id);
  if (!words) return fail(ctx, C2F_EINVAL, "words is NULL");
  int rc = sim_ready(ctx, *s);
  if (rc) return rc;
  CK(cudaSetDevice(ctx->device));
  const size_t bytes = (size_t)s->p.n_replicas * s->rows * s->wpr * 4;
  CK(cudaMemcpyAsync(words, s->ign_plane.p, bytes, cudaMemcpyDeviceToHost, ctx->read_stream));
  CK(cudaStreamSynchronize(ctx->read_stream));
  return C2F_OK;
}

C2F_API int c2f_get_scars_at_hour(c2f_ctx *ctx, int32_t sim_id, int32_t hour, uint8_t *scars) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto s = find_sim(ctx, sim_id);
  if (!s) return fail(ctx, C2F_ENOTFOUND, "unknown simulation %d", sim_id);
  if (!scars) return fail(ctx, C2F_EINVAL, "scars is NULL");
  int rc = sim_ready(ctx, *s);
  if (rc) return rc;
  if (!s->ign_step.p)
    return fail(ctx, C2F_EINVAL, "simulation did not keep ignition steps (C2F_OUT_IGN_STEPS)");
  if (hour < 0 || hour >= s->p.hours) return fail(ctx, C2F_EINVAL, "hour out of range");
  CK(cudaSetDevice(ctx->device));
  const int64_t total = (int64_t)s->n * s->p.n_replicas;
  const int32_t smax = (hour + 1) * (60 / s->p.minutes_per_step);
  cudaStream_t st = ctx->read_stream;
  DevBuf tmp;
  if ((rc = dalloc_on(ctx, tmp, (size_t)total, st))) return rc;
  k_scar_at_step<<<grid1(total, 256), 256, 0, st>>>(s->ign_step.as<int32_t>(), total, smax, tmp.as<uint8_t>());
  CKL("k_scar_at_step");
  CK(cudaMemcpyAsync(scars, tmp.p, (size_t)total, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return C2F_OK;
}

}  // extern "C"

namespace {

constexpr int32_t kCompareMaxHours = 8192;   // 3 H counters in shared memory

// Sec. 4.1 metrics of two finished simulations on st: hourly MSE / SSIM
// ([R][H], from the ignition steps) and the final scars' norm ([R], from the
// bit planes) into device memory.
int compare_launch(c2f_ctx *ctx, int32_t sim_x, int32_t sim_y, double *mse, double *ssim,
                   double *dnorm, cudaStream_t st) {
  auto X = find_sim(ctx, sim_x), Y = find_sim(ctx, sim_y);
  if (!X || !Y) return fail(ctx, C2F_ENOTFOUND, "unknown simulation %d", !X ? sim_x : sim_y);
  int rc;
  if ((rc = sim_ready(ctx, *X)) || (rc = sim_ready(ctx, *Y))) return rc;
  if (X->rows != Y->rows || X->cols != Y->cols || X->p.n_replicas != Y->p.n_replicas)
    return fail(ctx, C2F_EINVAL, "simulations differ in grid shape or replica count");
  const int32_t R = X->p.n_replicas;
  if (mse || ssim) {
    if (!X->ign_step.p || !Y->ign_step.p)
      return fail(ctx, C2F_EINVAL, "hourly metrics need ignition steps (C2F_OUT_IGN_STEPS) in both");
    if (X->p.hours != Y->p.hours || X->p.minutes_per_step != Y->p.minutes_per_step)
      return fail(ctx, C2F_EINVAL, "simulations differ in hours or minutes_per_step");
    if (X->p.hours > kCompareMaxHours) return fail(ctx, C2F_EINVAL, "at most %d hours", kCompareMaxHours);
    if (X->n < 2) return fail(ctx, C2F_EINVAL, "SSIM needs at least 2 cells");
  }
  CK(cudaSetDevice(ctx->device));
  if (mse || ssim) {
    const int32_t H = X->p.hours;
    const size_t smem = sizeof(uint32_t) * 3 * (size_t)H;
    if (smem > 48 * 1024) CK(cudaFuncSetAttribute(k_compare_hours, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)smem));
    k_compare_hours<<<R, 128, smem, st>>>(X->ign_step.as<int32_t>(), Y->ign_step.as<int32_t>(), X->n,
                                          60 / X->p.minutes_per_step, H, mse, ssim, dnorm);
    CKL("k_compare_hours");
  } else if (dnorm) {   // no hourly metrics asked for: the final scars' bit planes
    k_compare_final<<<R, 256, 0, st>>>(X->ign_plane.as<uint32_t>(), Y->ign_plane.as<uint32_t>(),
                                       (int64_t)X->rows * X->wpr, dnorm);
    CKL("k_compare_final");
  }
  if ((rc = note_read(ctx, *X, st))) return rc;
  return note_read(ctx, *Y, st);
}

}  // namespace

extern "C" {

C2F_API int c2f_compare_scars(c2f_ctx *ctx, int32_t sim_x, int32_t sim_y, double *mse, double *ssim,
                              double *dnorm) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto X = find_sim(ctx, sim_x);
  if (!X) return fail(ctx, C2F_ENOTFOUND, "unknown simulation %d", sim_x);
  const size_t RH = (size_t)X->p.n_replicas * X->p.hours, R = (size_t)X->p.n_replicas;
  cudaStream_t st = ctx->read_stream;
  DevBuf dm, ds, dd;
  int rc;
  if (mse && (rc = dalloc_on(ctx, dm, RH * 8, st))) return rc;
  if (ssim && (rc = dalloc_on(ctx, ds, RH * 8, st))) return rc;
  if (dnorm && (rc = dalloc_on(ctx, dd, R * 8, st))) return rc;
  if ((rc = compare_launch(ctx, sim_x, sim_y, dm.as<double>(), ds.as<double>(), dd.as<double>(), st)))
    return rc;
  if (mse) CK(cudaMemcpyAsync(mse, dm.p, RH * 8, cudaMemcpyDeviceToHost, st));
  if (ssim) CK(cudaMemcpyAsync(ssim, ds.p, RH * 8, cudaMemcpyDeviceToHost, st));
  if (dnorm) CK(cudaMemcpyAsync(dnorm, dd.p, R * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return C2F_OK;
}

C2F_API int c2f_compare_scars_device(c2f_ctx *ctx, int32_t sim_x, int32_t sim_y, double *mse_dev,
                                     double *ssim_dev, double *dnorm_dev) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  return compare_launch(ctx, sim_x, sim_y, mse_dev, ssim_dev, dnorm_dev, ctx->stream);
}

C2F_API int c2f_get_counters(c2f_ctx *ctx, int32_t sim_id, int64_t *work, int32_t *ignited,
                             int32_t *ign_cell) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto s = find_sim(ctx, sim_id);
  if (!s) return fail(ctx, C2F_ENOTFOUND, "unknown simulation %d", sim_id);
  int rc = sim_ready(ctx, *s);
  if (rc) return rc;
  CK(cudaSetDevice(ctx->device));
  const size_t R = (size_t)s->p.n_replicas;
  cudaStream_t st = ctx->read_stream;
  if (work) CK(cudaMemcpyAsync(work, s->work.p, R * 8, cudaMemcpyDeviceToHost, st));
  if (ignited) CK(cudaMemcpyAsync(ignited, s->n_ignited.p, R * 4, cudaMemcpyDeviceToHost, st));
  if (ign_cell) CK(cudaMemcpyAsync(ign_cell, s->ign_cell.p, R * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return C2F_OK;
}

C2F_API int c2f_get_scenarios(c2f_ctx *ctx, int32_t sim_id, int32_t *scenario) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto s = find_sim(ctx, sim_id);
  if (!s) return fail(ctx, C2F_ENOTFOUND, "unknown simulation %d", sim_id);
  if (!scenario) return fail(ctx, C2F_EINVAL, "scenario is NULL");
  int rc = sim_ready(ctx, *s);
  if (rc) return rc;
  const size_t R = (size_t)s->p.n_replicas;
  if (!s->scen.p) {   // one weather stream: every replica ran scenario 0
    std::memset(scenario, 0, R * 4);
    return C2F_OK;
  }
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->read_stream;
  CK(cudaMemcpyAsync(scenario, s->scen.p, R * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return C2F_OK;
}

C2F_API int c2f_set_list_capacity(c2f_ctx *ctx, int64_t cap) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  if (cap < 0 || cap > (1LL << 31)) return fail(ctx, C2F_EINVAL, "capacity out of range");
  ctx->cap_override = cap;
  return C2F_OK;
}

C2F_API int c2f_get_replica_profile(c2f_ctx *ctx, int32_t sim_id, int64_t *counters) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto s = find_sim(ctx, sim_id);
  if (!s) return fail(ctx, C2F_ENOTFOUND, "unknown simulation %d", sim_id);
  if (!counters) return fail(ctx, C2F_EINVAL, "counters is NULL");
  int rc = sim_ready(ctx, *s);
  if (rc) return rc;
  if (!s->prof.p) return fail(ctx, C2F_EINVAL, "the simulation ran without per-replica counters");
  CK(cudaSetDevice(ctx->device));
  CK(cudaMemcpyAsync(counters, s->prof.p, 8 * kProfCounters * (size_t)s->p.n_replicas, cudaMemcpyDeviceToHost,
                     ctx->read_stream));
  CK(cudaStreamSynchronize(ctx->read_stream));
  return C2F_OK;
}

C2F_API int c2f_serving_stats(c2f_ctx *ctx, int64_t *epochs, int64_t *admission_waits, int32_t *queued,
                              int32_t *running) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  if (epochs) *epochs = ctx->epochs_launched;
  if (admission_waits) *admission_waits = ctx->admission_waits;
  if (queued) *queued = (int32_t)ctx->pending.size();
  if (running) *running = (int32_t)ctx->inflight.size();
  return C2F_OK;
}

C2F_API int c2f_set_wait_limit(c2f_ctx *ctx, int64_t polls) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  if (polls < 0 || polls > 0xFFFFFFFFLL) return fail(ctx, C2F_EINVAL, "wait limit out of range");
  ctx->wait_limit = (uint32_t)polls;
  return C2F_OK;
}

C2F_API int c2f_test_hold_chunk(c2f_ctx *ctx, int32_t landscape_id, int32_t scenario, int32_t hour,
                                int32_t cell) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  auto L = find_land(ctx, landscape_id);
  if (!L) return fail(ctx, C2F_ENOTFOUND, "unknown landscape %d", landscape_id);
  if (!L->table || L->table->eager) return fail(ctx, C2F_EINVAL, "the landscape has no lazy table");
  const Table &T = *L->table;
  if (scenario < 0 || scenario >= T.n_scen || hour < 0 || hour >= T.key.hours || cell < 0 || cell >= L->n)
    return fail(ctx, C2F_EINVAL, "scenario, hour or cell out of range");
  CK(cudaSetDevice(ctx->device));
  const int32_t row = (int32_t)(cell / L->cols), col = (int32_t)(cell % L->cols);
  const size_t idx = ((size_t)scenario * T.key.hours + (size_t)hour) * (size_t)L->rows * L->wpr +
                     (size_t)row * L->wpr + (size_t)(col >> 5);
  static const uint32_t kBeingComputed = 1u;
  CK(cudaMemcpyAsync(T.chunk_state.as<uint32_t>() + idx, &kBeingComputed, 4, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return C2F_OK;
}

C2F_API int c2f_set_frontier_config(c2f_ctx *ctx, int threads, int64_t smem) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  if (threads != 32 && threads != 64 && threads != 128)
    return fail(ctx, C2F_EINVAL, "threads must be 32, 64 or 128 (one replica per warp)");
  if (smem < 0 || smem > 16) return fail(ctx, C2F_EINVAL, "smem must lie in [0, 16]");
  ctx->frontier_threads = threads;
  ctx->window_smem = smem != 0;
  ctx->warps_per_sm = smem >= 2 ? (int)smem : 0;
  return C2F_OK;
}

C2F_API int c2f_set_table_mode(c2f_ctx *ctx, int eager) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  ctx->eager_tables = eager != 0;
  return C2F_OK;
}

C2F_API int c2f_set_serving(c2f_ctx *ctx, int32_t max_inflight, int64_t max_epoch_replicas,
                            int64_t hbm_reserve_bytes) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  if (max_inflight < 1 || max_inflight > 16 || max_epoch_replicas < 1 || hbm_reserve_bytes < 0)
    return fail(ctx, C2F_EINVAL, "bad serving limits");
  ctx->max_inflight = max_inflight;
  ctx->max_epoch_replicas = max_epoch_replicas;
  ctx->hbm_reserve = hbm_reserve_bytes;
  return C2F_OK;
}

C2F_API int c2f_kernel_times(c2f_ctx *ctx, double *ms, int64_t *launches);

C2F_API int c2f_set_compaction(c2f_ctx *ctx, int32_t eighths) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  if (eighths < 2 || eighths > 7) return fail(ctx, C2F_EINVAL, "compaction trigger must be 2..7 eighths");
  ctx->compact_eighths = eighths;
  return C2F_OK;
}

// Launch-shape autotuner: coordinate descent over the frontier's knobs on a
// scaled-down copy of the mix (the same landscapes and options, replicas cut
// in proportion), each candidate timed by the frontier's kernel events:
//   1. warps per CTA x shared / global lists (threads 32, 64, 128 with
//      windowed shared-memory lists; 32, 128 with global lists);
//   2. shared-memory sizing (warps per SM the per-warp share is cut for:
//      the launch's own, 4, 6, 8, 11), with shared-memory lists only;
//   3. the compaction trigger (4, 6, 7 eighths of the list capacity);
//   4. the initial list capacity (automatic, 2x, 4x: fewer overflow re-runs
//      against more memory), with global lists only.
// The best setting of each stage is kept for the next; the winner stays on
// the context.  Results never depend on any of these.
C2F_API int c2f_autotune_full(c2f_ctx *ctx, int32_t n, const int32_t *landscape_ids,
                              const c2f_sim_params *params, int32_t sample_replicas, c2f_tuning *out) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  if (n < 1 || !landscape_ids || !params || sample_replicas < 1)
    return fail(ctx, C2F_EINVAL, "bad autotune arguments");
  int64_t total = 0;
  for (int32_t i = 0; i < n; ++i) total += std::max(params[i].n_replicas, 1);
  std::vector<c2f_sim_params> q(params, params + n);
  int64_t auto_cap = 0;
  for (int32_t i = 0; i < n; ++i) {   // the same mix of simulations, scaled down
    const int64_t r = (int64_t)params[i].n_replicas * sample_replicas / std::max<int64_t>(total, 1);
    q[i].n_replicas = (int32_t)std::max<int64_t>(1, std::min<int64_t>(r, params[i].n_replicas));
    q[i].outputs = C2F_OUT_SCARS | C2F_OUT_COUNTERS;
    auto L = find_land(ctx, landscape_ids[i]);
    if (!L) return fail(ctx, C2F_ENOTFOUND, "unknown landscape %d", landscape_ids[i]);
    auto_cap = std::max(auto_cap, std::max<int64_t>(1024, 2 * (int64_t)(L->rows + L->cols)));
  }
  struct Knobs { int threads; bool win; int warps_per_sm; int eighths; int64_t cap; };
  const Knobs keep{ctx->frontier_threads, ctx->window_smem, ctx->warps_per_sm, ctx->compact_eighths,
                   ctx->cap_override};
  const bool keep_prof = ctx->profiling, keep_rc = ctx->replica_counters;
  auto apply = [&](const Knobs &k) {
    ctx->frontier_threads = k.threads; ctx->window_smem = k.win; ctx->warps_per_sm = k.warps_per_sm;
    ctx->compact_eighths = k.eighths; ctx->cap_override = k.cap;
  };
  std::vector<int32_t> sids(n);
  int32_t tried = 0;
  auto time_of = [&](const Knobs &k, double *ms_out) -> int {
    apply(k);
    ctx->profiling = true;
    ctx->replica_counters = false;
    double ms[C2F_KT_FAMILIES];
    int64_t cnt[C2F_KT_FAMILIES];
    int rc = c2f_kernel_times(ctx, ms, cnt);   // reset
    if (!rc) rc = simulate_many(ctx, n, landscape_ids, q.data(), sids.data());
    if (!rc) rc = c2f_kernel_times(ctx, ms, cnt);
    if (!rc) for (int32_t i = 0; i < n; ++i) ctx->sims.erase(sids[i]);
    ++tried;
    *ms_out = ms[2];
    return rc;
  };
  auto restore = [&]() { apply(keep); ctx->profiling = keep_prof; ctx->replica_counters = keep_rc; };
  Knobs best{32, true, 0, 6, 0};
  double best_ms = 1e300;
  // after the launch shapes, a candidate replaces the incumbent only when it is
  // at least 3 % faster: smaller differences are within the sample's timing noise,
  // and keeping the incumbent makes repeated tunings of one mix agree
  constexpr double kMargin = 0.97;
  // 1. warps per CTA x shared / global lists
  const Knobs shapes[5] = {{32, true, 0, 6, 0}, {64, true, 0, 6, 0}, {128, true, 0, 6, 0},
                           {32, false, 0, 6, 0}, {128, false, 0, 6, 0}};
  for (const Knobs &k : shapes) {
    double ms;
    if (int rc = time_of(k, &ms)) { restore(); return rc; }
    if (ms < best_ms) { best_ms = ms; best = k; }
  }
  // 2. shared-memory sizing (shared-memory lists only)
  if (best.win) {
    const Knobs base = best;
    for (int wps : {4, 6, 8, 11}) {
      Knobs k = base;
      k.warps_per_sm = wps;
      double ms;
      if (int rc = time_of(k, &ms)) { restore(); return rc; }
      if (ms < kMargin * best_ms) { best_ms = ms; best = k; }
    }
  }
  // 3. compaction trigger
  {
    const Knobs base = best;
    for (int e : {4, 7}) {
      Knobs k = base;
      k.eighths = e;
      double ms;
      if (int rc = time_of(k, &ms)) { restore(); return rc; }
      if (ms < kMargin * best_ms) { best_ms = ms; best = k; }
    }
  }
  // 4. initial list capacity (global lists only; shared lists are sized by stage 2)
  if (!best.win) {
    const Knobs base = best;
    for (int64_t mult : {2, 4}) {
      Knobs k = base;
      k.cap = auto_cap * mult;
      double ms;
      if (int rc = time_of(k, &ms)) { restore(); return rc; }
      if (ms < kMargin * best_ms) { best_ms = ms; best = k; }
    }
  }
  apply(best);
  ctx->profiling = keep_prof;
  ctx->replica_counters = keep_rc;
  if (out) {
    out->threads = best.threads;
    out->smem_lists = best.win ? 1 : 0;
    out->warps_per_sm = best.warps_per_sm;
    out->compact_eighths = best.eighths;
    out->list_capacity = best.cap;
    out->frontier_ms = best_ms;
    out->candidates = tried;
  }
  return C2F_OK;
}

C2F_API int c2f_autotune(c2f_ctx *ctx, int32_t n, const int32_t *landscape_ids,
                         const c2f_sim_params *params, int32_t sample_replicas, int32_t *best_threads,
                         int32_t *best_smem, double *best_ms) {
  c2f_tuning t{};
  const int rc = c2f_autotune_full(ctx, n, landscape_ids, params, sample_replicas, &t);
  if (rc) return rc;
  if (best_threads) *best_threads = t.threads;
  if (best_smem) *best_smem = t.smem_lists ? (t.warps_per_sm >= 2 ? t.warps_per_sm : 1) : 0;
  if (best_ms) *best_ms = t.frontier_ms;
  return C2F_OK;
}

C2F_API int c2f_profile(c2f_ctx *ctx, int enable) {
  if (!ctx) return C2F_EINVAL;
  if (enable & ~(C2F_PROFILE_KERNELS | C2F_PROFILE_REPLICAS)) return C2F_EINVAL;
  LOCK;
  ctx->profiling = (enable & C2F_PROFILE_KERNELS) != 0;
  ctx->replica_counters = (enable & C2F_PROFILE_REPLICAS) != 0;
  return C2F_OK;
}

C2F_API int c2f_trace(c2f_ctx *ctx, uint64_t *records_dev, int64_t capacity) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  if (records_dev && capacity <= 0) return fail(ctx, C2F_EINVAL, "trace capacity must be positive");
  if (!records_dev && capacity != 0) return fail(ctx, C2F_EINVAL, "no trace buffer but a capacity");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  if (records_dev) {
    int rc;
    // the cursor lives on the context's own stream, which outlives any caller stream
    if (!ctx->trace_cursor.p && (rc = dalloc_on(ctx, ctx->trace_cursor, 8, ctx->own_stream))) return rc;
    CK(cudaMemsetAsync(ctx->trace_cursor.p, 0, 8, ctx->own_stream));
    CK(cudaStreamSynchronize(ctx->own_stream));
  }
  ctx->trace_rec = reinterpret_cast<unsigned long long *>(records_dev);
  ctx->trace_cap = records_dev ? capacity : 0;
  return C2F_OK;
}

C2F_API int c2f_trace_count(c2f_ctx *ctx, int64_t *count) {
  if (!ctx || !count) return C2F_EINVAL;
  LOCK;
  *count = 0;
  if (!ctx->trace_cursor.p) return C2F_OK;
  CK(cudaSetDevice(ctx->device));
  unsigned long long v = 0;
  CK(cudaMemcpyAsync(&v, ctx->trace_cursor.p, 8, cudaMemcpyDeviceToHost, ctx->read_stream));
  CK(cudaStreamSynchronize(ctx->read_stream));
  *count = (int64_t)v;
  return C2F_OK;
}

C2F_API int c2f_fp64_peak(c2f_ctx *ctx, double *gflops) {
  if (!ctx || !gflops) return C2F_EINVAL;
  LOCK;
  CK(cudaSetDevice(ctx->device));
  const int32_t iters = 4096;
  const unsigned blocks = (unsigned)ctx->sm_count * 8, threads = 256;
  DevBuf sink;
  int rc;
  if ((rc = dalloc(ctx, sink, sizeof(double) * blocks))) return rc;
  cudaEvent_t a = get_event(ctx), b = get_event(ctx);
  if (!a || !b) return fail(ctx, C2F_ECUDA, "no CUDA event");
  double best = 0.0;
  for (int rep = 0; rep < 4; ++rep) {   // the first launch warms up; the best of the rest counts
    CK(cudaEventRecord(a, ctx->stream));
    k_dfma_peak<<<blocks, threads, 0, ctx->stream>>>(sink.as<double>(), iters);
    CKL("k_dfma_peak");
    CK(cudaEventRecord(b, ctx->stream));
    CK(cudaEventSynchronize(b));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, a, b));
    const double flop = 2.0 * 8.0 * iters * (double)blocks * threads;
    if (rep > 0 && ms > 0.0f) best = std::max(best, flop / (ms * 1e-3) / 1e9);
  }
  ctx->event_pool.push_back(a);
  ctx->event_pool.push_back(b);
  *gflops = best;
  return C2F_OK;
}

C2F_API int c2f_kernel_times(c2f_ctx *ctx, double *ms, int64_t *launches) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  for (auto &E : ctx->inflight) CK(cudaStreamSynchronize(E->stream));
  for (int f = 0; f < C2F_KT_FAMILIES; ++f) {
    double tot = 0.0;
    for (auto &pr : ctx->prof_events[f]) {
      float t = 0.0f;
      if (cudaEventElapsedTime(&t, pr.first, pr.second) == cudaSuccess) tot += t;
      else cudaGetLastError();
      ctx->event_pool.push_back(pr.first);
      ctx->event_pool.push_back(pr.second);
    }
    if (ms) ms[f] = tot;
    if (launches) launches[f] = (int64_t)ctx->prof_events[f].size();
    ctx->prof_events[f].clear();
  }
  return C2F_OK;
}

C2F_API int c2f_release(c2f_ctx *ctx, int32_t id) {
  if (!ctx) return C2F_EINVAL;
  LOCK;
  CK(cudaSetDevice(ctx->device));
  auto s = find_sim(ctx, id);
  if (s) {
    if (s->state == S_PENDING) {
      auto it = std::find(ctx->pending.begin(), ctx->pending.end(), s);
      if (it != ctx->pending.end()) ctx->pending.erase(it);
      s->state = S_CANCELED;
    } else if (s->state == S_RUNNING) {
      s->cancel_requested = true;   // the epoch still holds it until it finishes
    }
    ctx->sims.erase(id);
    return C2F_OK;
  }
  if (ctx->lands.erase(id)) return C2F_OK;   // simulations holding it keep it alive
  return fail(ctx, C2F_ENOTFOUND, "unknown id %d", id);
}

}  // extern "C"
