// c2f_layout.cuh -- data layout shared by the kernels (c2f_kernels.cu) and the
// host runtime (c2f_runtime.cu); no device code.
#pragma once
#include <cstdint>


namespace c2f {

struct MathConstants {
  double inv_fact[24];   // 1/k!
  double log_c[12];      // 1/(2n+1)
  double sin_c[10];      // (-1)^n/(2n+1)!
  double cos_c[10];      // (-1)^n/(2n)!
  float inv_fact_f[12];
  float log_cf[8];
  float sin_cf[8];
  float cos_cf[8];
};

enum FuelCode : int {
  F_NONE = 0, F_C1, F_C2, F_C3, F_C4, F_C5, F_C6, F_C7, F_D1, F_M1, F_M2,
  F_O1A, F_O1B, F_S1, F_S2, F_S3, F_NCODES
};

struct FuelCoef {
  double a, b, c, q, bui0;
  double inv_c, neg_inv_b;   // RN(1/c), RN(-1/b); 0 when c / b = 0
  int32_t c2, inv_c2;        // 2c and 2/c when they are small integers (half-integer powers), else 0
};

struct HourPrep {
  double ws, ff, isz, sin_w, cos_w;
  double cf;              // O1 curing factor
  double be[F_NCODES];    // build-up effect per fuel code
  double rszf[F_NCODES];  // RSI at zero wind and slope per code (O1 includes curing)
  double inv_a[F_NCODES]; // RN(1 / (a mult)) of each code's own curve (mult = curing for O1, else 1)
  double inv_a_d1m2;      // RN(1 / (a_D1 0.2)), the D1 part of M2
  double inv_isz;         // RN(1 / ISZ)
  double wsx_w, wsy_w;    // RN(WS sin WAZ), RN(WS cos WAZ): the wind's part of the net vector
  int32_t pos;            // 1: every fuel's HROS this hour is > 1e-200 (a lower bound says so)
};

struct CellPrep { double sf, sin_s, cos_s; };

// One simulation inside a frontier launch (several for a batch).
// Launch trace (c2f_trace): one record per K1 CTA and per frontier replica,
// four u64 each: kind | SM id << 8 | aux << 32, tag, start and end in
// nanoseconds of the global timer.  rec == nullptr: off.
struct TraceArgs {
  unsigned long long *rec;      // [cap][4]
  unsigned long long *cursor;   // records claimed so far (only the first cap are written)
  long long cap;
  long long tag;                // K1: the table's build number (frontier jobs carry their own)
};
constexpr uint32_t kTraceTable = 1, kTraceReplica = 2;

struct SimJob {
  // landscape
  int32_t rows, cols, wpr;        // wpr: 32-bit words per row of a bit plane
  int32_t n_burnable;
  const uint32_t *burnable;       // rows*wpr words, bit = burnable and not harvested
  const int32_t *burnable_list;   // burnable cell ids in row-major order
  // rate-of-spread table of this run
  int64_t *base;                  // [hours][N][8] fixed-point per-period increments
  double *hros;                   // [hours][N]
  // Rows of the table are filled on demand, 32 cells (one bit-plane word) at a
  // time, when chunk_state is set: [hours][rows*wpr], 0 empty, 1 being
  // computed, >= 2 done.  nullptr: every row is present.
  uint32_t *chunk_state;
  const HourPrep *hour;           // [hours], or nullptr (no positivity shortcut)
  const uint8_t *fuel;            // FBP inputs of the on-demand rows
  const float *slope;             // nullable
  const CellPrep *cell;
  double pcf, const_ros, const_bros, const_lb, dt2p32;
  int32_t ellipse_mode;
  // weather scenarios (Sec. 3.1, uncertainty (3)): with n_scen > 1 the table
  // holds n_scen stacked tables ([n_scen][scen_hours] rows of base / hros /
  // chunk_state, [n_scen][prep_hours] hour preps); replica r draws scen[r]
  // (K2) and the frontier reads that scenario's rows
  int32_t n_scen, scen_hours, prep_hours;
  const uint64_t *scen_thr;       // [n_scen] thresholds T_s (T_{S-1} = 2^32)
  int32_t *scen;                  // [R] drawn scenario per replica
  // run parameters
  uint64_t seed;
  float sigma;
  int32_t ignition_mode, ignition_cell;
  double thr, delta;
  int32_t recv_gate;              // receive_gate(thr, const_ros): when receive tests are needed
  int32_t sph, hours;             // fire periods per hour, simulated hours
  int32_t burn_min, burn_max;     // burning hours per day {min..max}; 0, 0: no limit
  int64_t d_orth, d_diag;         // axis lengths in fixed point
  int32_t n_replicas;
  // per-replica outputs
  uint32_t *ign_plane;            // [R][rows*wpr] scar bits
  int32_t *ign_step;              // [R][N] or nullptr
  int64_t *work;                  // [R]
  int32_t *n_ignited;             // [R]
  int32_t *ign_cell;              // [R]
  long long *prof;                // [R][kProfCounters] per-replica profile counters, or nullptr (off)
  long long trace_tag;            // the simulation's creation number, for trace records
  int32_t *status;                // [R] 0 ok, 1 list capacity exceeded, 2 internal error,
                                  //     3 ignition cell outside the grid or not burnable,
                                  //     4 a bounded wait (for a lazy table chunk) ran out
};

struct FrontierArgs {
  const SimJob *jobs;
  int32_t n_jobs;
  const int64_t *item_begin;      // [n_jobs + 1]: replicas of job j are items item_begin[j]..
  const int64_t *item_list;       // nullptr: items 0..n_items-1; else explicit global items
  int64_t n_items;
  unsigned long long *counter;    // work-list cursor (zeroed before the launch)
  int32_t cap;                    // burning-list capacity per slot
  int32_t *ent_cell;              // [slots][cap] cell as row << 16 | col
  int32_t *ent_link;              // [slots][cap] next entry in the same calendar list (-1 none)
  uint8_t *ent_cofs;              // [slots][cap][8] per-axis crossing offsets this hour
                                  //   (0xFE open axis, no crossing this hour; 0xFF closed)
  int64_t *ent_P;                 // [slots][cap][8] progress at the start of the next hour
  int64_t pw_max;                 // words per bit plane of the largest landscape
  uint32_t *brn_scratch;          // [slots][pw_max] Burned planes
  uint32_t *avail_scratch;        // [slots][pw_max] Available planes (global-plane variant)
  int64_t smem_warp_words;        // 32-bit words of dynamic shared memory per warp
  uint32_t wait_limit;            // polls before a wait for a table chunk gives up; 0 = default
  int32_t compact_at;             // list entries above which the list is compacted within an
                                  //   hour (0 = three quarters of cap)
  TraceArgs trace;                // one record per replica when on
};

// K1 launch arguments: grid.y covers hours hour0 .. hour0 + gridDim.y - 1
struct RosTableArgs {
  const uint8_t *fuel;
  const float *slope;
  const uint32_t *burnable;
  int32_t rows, cols, wpr;
  const CellPrep *cell;
  const HourPrep *hour;    // indexed by absolute hour
  int32_t hour0;
  double pcf, const_ros, const_bros, const_lb, dt2p32;
  int32_t ellipse_mode;
  int64_t *base;           // [hour][N][8] (absolute hour), or nullptr
  double *hros;            // [hour][N], or nullptr
  double *ros8;            // export: [N][8] of hour0 only, or nullptr
  const int32_t *order;    // cells grouped by (fuel code, sloped); nullptr = identity
  TraceArgs trace;         // one record per CTA when on
};

// When the frontier needs the receive test of Sec. 3.1 (HROS * f > threshold),
// decided on the host from the threshold and the constant-ROS setting so that
// the frontier's loops hold no binary64 compare: 0 never (threshold < 0: every
// message to an Available cell ignites it), 1 never (threshold 0 with a
// positive constant ROS), 2 only in hours whose lower bound on every fuel's
// HROS is not positive (threshold 0), 3 always (threshold > 0, or NaN)
inline int32_t receive_gate(double thr, double const_ros) {
  if (thr < 0.0) return 0;
  if (thr == 0.0) return const_ros > 0.0 ? 1 : 2;
  return 3;
}

constexpr int kOrderBuckets = 2 * 16;   // (fuel code, slope > 0); code 0 = not burnable

constexpr uint8_t kNone = 0xFF;
constexpr int kProfCounters = 16;   // per-replica frontier profile counters (c2f_get_replica_profile)
// shared-memory window of the per-replica bit planes: kWinRows x (32 kWinWords) cells
constexpr int kWinRows = 256;
constexpr int kWinWords = 8;

}  // namespace c2f
