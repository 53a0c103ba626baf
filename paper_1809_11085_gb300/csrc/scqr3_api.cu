// scqr3_api.cu -- the C ABI of include/scqr3.h: argument checks, workspace
// layout and the launch sequence of one factorization.
//
// A factorization is a fixed sequence of kernels on one stream, with no host
// synchronization: the number of passes is decided on the device (the
// Cholesky kernel of pass k sets flags that later launches read), so kernels
// of passes that turn out not to be needed return at once. That keeps a call
// capturable in a CUDA graph and free of host round trips.
#include <cstdint>
#include <cstring>
#include <atomic>
#include <cstdio>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "scqr3_internal.cuh"

namespace scqr3 {
cudaError_t pass_setup(int np, int* ctas_per_sm, PassGeom* geo);
void launch_pass(int np, int grid, cudaStream_t s, const double* src, int64_t lds, double* dst,
                 int64_t ldd, const Params& P, int pass, const double* rk, const double* lt,
                 double* partials, int part_stride, DevState* st);
void launch_reduce(cudaStream_t s, const double* partials, int n_partials, int stride, double* out,
                   const DevState* st, int pass);
void launch_chol(int np, cudaStream_t s, const Params& P, int pass, const double* gram,
                 double* rstack, double* racc, double* Rout, double* Rpass, DevState* st,
                 scqr3_info* info);
void launch_bfactor(cudaStream_t s, int bs, const double* B, int64_t nblk, double* lt, DevState* st,
                    int sms);
cudaError_t n256_setup(int* trsm_per_sm, int* gram_per_sm);
void launch_trsm256(int grid, cudaStream_t s, const double* src, int64_t lds, double* dst, int64_t ldd,
                    const Params& P, int pass, const double* rk, const DevState* st);
void launch_gram256(int grid, cudaStream_t s, const double* src, int64_t lds, const Params& P, int pass,
                    double* partials, int part_stride, const DevState* st);
void launch_chol256(cudaStream_t s, const Params& P, int pass, const double* gram, double* rstack,
                    double* racc, double* Rout, double* Rpass, DevState* st, scqr3_info* info, double* S,
                    double* Ra);
cudaError_t df_setup();
cudaError_t df_occupancy(int np, int* per_sm);
int df_groups(int np);
int df_rows_per_panel(int np);
void launch_df_finish(int grid, cudaStream_t s, double* Q, int64_t ldq, int64_t m, int n,
                      int max_passes, const DevState* st);
void launch_df_pass(int np, int grid, cudaStream_t s, const double* src, int64_t lds, double* dst,
                    int64_t ldd, const Params& P, int pass, const double* rk, double* partials,
                    int part_stride, DevState* st);
cudaError_t csr_setup(int per_sm[4]);
int csr_rows_per_panel(int np);
int csr_groups(int np);
void launch_csr_check(int grid, cudaStream_t s, int64_t m, const scqr3_B* B, DevState* st);
void launch_csr_gram(int np, int grid, cudaStream_t s, const double* src, int64_t lds, const Params& P,
                     int pass, const scqr3_B* B, double* partials, int part_stride, const DevState* st);
cudaError_t tc_setup();
int tc_grid(int64_t m, int np, int sms);
cudaError_t tc_solve_setup();
void launch_tc_split_r(cudaStream_t s, const double* rk, int np, int n, int w, int pass, const DevState* st,
                       double* rdiag);
void launch_tc_update(int sms, cudaStream_t s, int k, const double* y, int64_t ldy, const double* x1,
                      int64_t ldx, double* q1, int64_t ldq, int64_t m, int n1, int pass, const double* rk, int np,
                      int r0, int c0, int ldb, int ky, DevState* st, long long wait_ns);
void launch_tc_gram(int grid, int sms, cudaStream_t s, const double* src, int64_t lds, const Params& P, int pass,
                    unsigned long long* colmax, double* partials, int part_stride, DevState* st, int pairs,
                    const double* lt, int64_t blk0, int scan, int offd_only);
cudaError_t tc_fused_setup();
bool tc_fused_supported(int n);
void launch_tc_fused(int sms, cudaStream_t s, const double* X, int64_t ldx, double* Q, int64_t ldq, const Params& P,
                     int pass, const double* rk, unsigned long long* colmax, DevState* st);
void launch_status(cudaStream_t s, const DevState* st, scqr3_info* info);

namespace {

// The tensor-core Gram works on blocks of 64 columns.
int tc_np(int n) { return n <= 64 ? 64 : n <= 128 ? 128 : 256; }

int padded_n(int n) {
  if (n <= 16) return 16;
  if (n <= 32) return 32;
  if (n <= 64) return 64;
  if (n <= 128) return 128;
  if (n <= 256) return 256;
  return 0;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Per-device, per-size launch geometry (occupancy query and shared-memory
// opt-in happen once).
struct DevGeo {
  bool ready = false;
  int sms = 0;
  int trsm256_per_sm = 0, gram256_per_sm = 0;
  int ctas_per_sm[5] = {0, 0, 0, 0, 0};
  int df_ctas_per_sm[5] = {0, 0, 0, 0, 0};
  int csr_ctas_per_sm[4] = {0, 0, 0, 0};
  PassGeom geo[5];
};
constexpr int kMaxDevices = 64;
DevGeo g_geo[kMaxDevices];
std::mutex g_mu;

int np_slot(int np) { return np == 16 ? 0 : np == 32 ? 1 : np == 64 ? 2 : np == 128 ? 3 : 4; }

cudaError_t device_geo(int np, int* grid_max, PassGeom* geo) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  DevGeo& d = g_geo[dev];
  if (!d.ready) {
    e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    for (int s : {16, 32, 64, 128}) {
      e = pass_setup(s, &d.ctas_per_sm[np_slot(s)], &d.geo[np_slot(s)]);
      if (e != cudaSuccess) return e;
      if (d.ctas_per_sm[np_slot(s)] < 1) return cudaErrorInvalidConfiguration;
    }
    e = n256_setup(&d.trsm256_per_sm, &d.gram256_per_sm);
    if (e != cudaSuccess) return e;
    if (d.trsm256_per_sm < 1 || d.gram256_per_sm < 1) return cudaErrorInvalidConfiguration;
    e = df_setup();
    if (e != cudaSuccess) return e;
    for (int s : {16, 32, 64, 128}) {
      e = df_occupancy(s, &d.df_ctas_per_sm[np_slot(s)]);
      if (e != cudaSuccess) return e;
      if (d.df_ctas_per_sm[np_slot(s)] < 1) return cudaErrorInvalidConfiguration;
    }
    e = csr_setup(d.csr_ctas_per_sm);
    if (e != cudaSuccess) return e;
    e = tc_setup();
    if (e != cudaSuccess) return e;
    e = tc_solve_setup();
    if (e != cudaSuccess) return e;
    e = tc_fused_setup();
    if (e != cudaSuccess) return e;
    for (int k = 0; k < 4; ++k)
      if (d.csr_ctas_per_sm[k] < 1) return cudaErrorInvalidConfiguration;
    d.ready = true;
  }
  if (np == 256) {
    // gram256: two roles of one CTA per SM each half; trsm256 sized separately
    *grid_max = d.sms * d.gram256_per_sm;
    *geo = PassGeom{256, 64, 1, kThreads, 4, 65, 0};
    return cudaSuccess;
  }
  *grid_max = d.sms * d.ctas_per_sm[np_slot(np)];
  *geo = d.geo[np_slot(np)];
  return cudaSuccess;
}

int trsm256_grid(int64_t m) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int64_t np = (m + 255) / 256;
  const int64_t g = (int64_t)g_geo[dev].sms * g_geo[dev].trsm256_per_sm;
  return (int)(np < g ? (np < 1 ? 1 : np) : g);
}

int csr_grid_max(int np) {
  int dev = 0;
  cudaGetDevice(&dev);
  return g_geo[dev].sms * g_geo[dev].csr_ctas_per_sm[np_slot(np)];
}

int df_grid_max(int np) {
  int dev = 0;
  cudaGetDevice(&dev);
  return g_geo[dev].sms * g_geo[dev].df_ctas_per_sm[np_slot(np)];
}

int sm_count() {
  int dev = 0;
  cudaGetDevice(&dev);
  return (dev >= 0 && dev < kMaxDevices && g_geo[dev].ready) ? g_geo[dev].sms : 1;
}

int check_args(int64_t m, int n, const scqr3_B* B, const scqr3_opts* opts, bool shard = false) {
  if (n < 1) return -3;
  if (shard ? m < 1 : m < n) return -2;  // a row block of a partitioned X may be shorter than n
  if (B && (B->bs != 0 && B->bs != 1 && B->bs != 2 && B->bs != 4 && B->bs != 8 && B->bs != 16))
    return -5;
  if (B && B->bs > 0 && ((m % B->bs) != 0 || !B->blocks)) return -5;
  // CSR form: arrays present, a diagonal entry per row possible, int32 columns
  if (B && B->bs == 0 && (!B->row_ptr || !B->col_idx || !B->vals || B->nnz < m || m > INT32_MAX))
    return -5;
  if (B && B->bs == 0 && n > 128) return SCQR3_E_UNSUPPORTED;
  if (opts && opts->max_passes != 0 && (opts->max_passes < 3 || opts->max_passes > SCQR3_MAX_PASSES))
    return -12;
  if (opts && opts->precision != SCQR3_PREC_FP64 && opts->precision != SCQR3_PREC_MIXED &&
      opts->precision != SCQR3_PREC_TC && opts->precision != SCQR3_PREC_MIXED_TC)
    return -12;
  const bool tcp = opts && (opts->precision == SCQR3_PREC_TC || opts->precision == SCQR3_PREC_MIXED_TC);
  // tensor-core Gram: at most 2^31 rows (its exact int64 digit-sum
  // accumulators); n <= 128, or n <= 256 for the FP64-accurate form with B = I
  if (tcp && (n > 256 || m > ((int64_t)1 << 31))) return SCQR3_E_UNSUPPORTED;
  if (tcp && n > 128 && (B || opts->precision != SCQR3_PREC_TC)) return SCQR3_E_UNSUPPORTED;
  // tensor-core forms with B: block-diagonal with blocks of 1, 2, 4 or 8 rows
  // (they divide the kernel's 8-row units), FP64 substitution only
  if (tcp && B && (B->bs == 0 || B->bs > 8 || opts->precision == SCQR3_PREC_MIXED_TC)) return SCQR3_E_UNSUPPORTED;
  if (opts && opts->precision == SCQR3_PREC_MIXED && B) return -5;  // mixed form: B = I only
  if (opts && opts->norm_x2 < 0.0 && B) return -12;  // the 2-norm estimate: B = I only
  if (opts && opts->algorithm != 0 && opts->algorithm != SCQR3_ALG_SCQR3 &&
      opts->algorithm != SCQR3_ALG_ADAPTIVE)
    return -12;
  if (padded_n(n) == 0) return SCQR3_E_UNSUPPORTED;
  // n > 128: FP64, B = I only
  if (n > 128 && (B || (opts && opts->precision == SCQR3_PREC_MIXED))) return SCQR3_E_UNSUPPORTED;
  return SCQR3_OK;
}

// Grid of the pass kernel and the workspace carve-up. The partial-slot area is
// sized for the largest of the FP64, mixed and tensor-core kernels' needs, so
// one workspace serves every precision.
// Host-buffer entry point: X arrives and Q leaves in row chunks of this size.
constexpr int kHostChunks = 8;
constexpr int64_t kHostMinChunkRows = 262144;
int64_t host_chunk_rows(int64_t m) {
  int64_t r = (m + kHostChunks - 1) / kHostChunks;
  r = (r + 255) / 256 * 256;
  return r < kHostMinChunkRows ? kHostMinChunkRows : r;
}

int make_layout_one(int64_t m, int n, const scqr3_B* B, int prec, int host_chunks, Layout* L, int* grid,
                    PassGeom* geo) {
  const bool mixed = prec == SCQR3_PREC_MIXED || prec == SCQR3_PREC_MIXED_TC;
  const bool tcg = prec == SCQR3_PREC_TC || prec == SCQR3_PREC_MIXED_TC;
  const int np = tcg ? tc_np(n) : padded_n(n);
  int grid_max = 0;
  if (device_geo(np, &grid_max, geo) != cudaSuccess) return SCQR3_E_CUDA;
  const int64_t npanels = (m + geo->pr - 1) / geo->pr;
  int grid64 = (int)(npanels < grid_max ? npanels : grid_max);
  if (grid64 < 1) grid64 = 1;
  if (np == 256) {
    grid64 = grid_max & ~1;  // two roles; even
    if (grid64 < 2) grid64 = 2;
  }
  const int df_max = np == 256 ? 1 : df_grid_max(np);
  const int64_t np_df = (m + df_rows_per_panel(np) - 1) / df_rows_per_panel(np);
  int griddf = (int)(np_df < df_max ? np_df : df_max);
  if (griddf < 1) griddf = 1;
  const int slots64 = grid64 * geo->groups, slotsdf = griddf * df_groups(np);
  *grid = mixed ? griddf : grid64;
  const int E = pk_size(np);
  L->part_stride = E + 1;
  L->n_partials = mixed ? slotsdf : slots64;
  int slots_alloc = slots64 > slotsdf ? slots64 : slotsdf;
  L->csr_grid = 0;
  if (B && B->bs == 0 && np <= 128) {
    const int64_t np_csr = (m + csr_rows_per_panel(np) - 1) / csr_rows_per_panel(np);
    const int csr_max = csr_grid_max(np);
    L->csr_grid = (int)(np_csr < csr_max ? np_csr : csr_max);
    if (L->csr_grid < 1) L->csr_grid = 1;
    L->n_partials = L->csr_grid * csr_groups(np);
    if (L->n_partials > slots_alloc) slots_alloc = L->n_partials;
  }
  const int sms = sm_count();
  // the tensor-core Gram's slots and column scales are always reserved, so
  // one workspace serves every precision of a shape
  {
    L->tc_grid = tc_grid(m, tcg ? np : (np <= 64 ? 64 : 128), sms);
    if (L->tc_grid > slots_alloc) slots_alloc = L->tc_grid;
    if (tcg) L->n_partials = L->tc_grid;
  }
  size_t off = 0;
  L->state = off;
  off = align256(off + sizeof(DevState));
  L->gram = off;
  off = align256(off + sizeof(double) * (E + 1));
  L->rstack = off;
  off = align256(off + sizeof(double) * (size_t)E * SCQR3_MAX_PASSES);
  L->racc = off;
  off = align256(off + sizeof(double) * E);
  L->chol = off;  // Cholesky work buffers in global memory (n > 128)
  if (np == 256) off = align256(off + sizeof(double) * 2 * (size_t)E);
  if (host_chunks && !B) {
    // the first Gram runs per chunk, each chunk into slots of its own (sized
    // for every precision, like the rest of the workspace)
    int f64 = 0, fdf = 0, ftc = 0;
    const int64_t cr = host_chunk_rows(m);
    for (int64_t r0 = 0; r0 < m; r0 += cr) {
      const int64_t rows = (m - r0) < cr ? (m - r0) : cr;
      ftc += tc_grid(rows, tcg ? np : (np <= 64 ? 64 : 128), sms);
      if (np == 256) {
        f64 += grid64;
      } else {
        const int64_t pdf = (rows + df_rows_per_panel(np) - 1) / df_rows_per_panel(np);
        fdf += (int)(pdf < griddf ? pdf : griddf) * df_groups(np);
        const int64_t pn = (rows + geo->pr - 1) / geo->pr;
        f64 += (int)(pn < grid64 ? pn : grid64) * geo->groups;
      }
    }
    const int first = f64 > fdf ? (f64 > ftc ? f64 : ftc) : (fdf > ftc ? fdf : ftc);
    if (first > slots_alloc) slots_alloc = first;
  }
  L->rdev = L->infodev = 0;
  if (host_chunks) {
    L->rdev = off;
    off = align256(off + sizeof(double) * (size_t)n * n);
    L->infodev = off;
    off = align256(off + sizeof(scqr3_info));
  }
  L->colmax = off;
  off = align256(off + sizeof(unsigned long long) * 256);
  L->tcr = off;
  off = align256(off + sizeof(double) * 8 * pk_size(32));
  L->lt = off;
  if (B && B->bs > 0) {
    const int64_t nblk = m / B->bs;
    off = align256(off + sizeof(double) * (size_t)nblk * (B->bs * (B->bs + 1) / 2));
  }
  L->partials = off;
  off = align256(off + sizeof(double) * (size_t)slots_alloc * L->part_stride);
  L->total = off;
  return SCQR3_OK;
}

// The layout for `prec`, with a total size that fits every precision the
// shape supports, so that one workspace serves them all.
int make_layout(int64_t m, int n, const scqr3_B* B, int prec, int host_chunks, Layout* L, int* grid,
                PassGeom* geo) {
  const int r = make_layout_one(m, n, B, prec, host_chunks, L, grid, geo);
  if (r != SCQR3_OK) return r;
  for (int p : {SCQR3_PREC_FP64, SCQR3_PREC_TC, SCQR3_PREC_MIXED_TC}) {
    const bool tc_ok = n <= 128 ? (!B || (p == SCQR3_PREC_TC && B->bs > 0 && B->bs <= 8))
                                : (n <= 256 && !B && p == SCQR3_PREC_TC);
    if (p == prec || (p != SCQR3_PREC_FP64 && !tc_ok)) continue;
    Layout L2;
    int g2;
    PassGeom geo2;
    if (make_layout_one(m, n, B, p, host_chunks, &L2, &g2, &geo2) == SCQR3_OK && L2.total > L->total)
      L->total = L2.total;
  }
  return SCQR3_OK;
}

// ---- launch timing -------------------------------------------------------------------------
struct Timer {
  std::mutex mu;
  bool on = false;
  int cap = 0;
  int used = 0;       // events used
  int launches = 0;   // launches seen (may exceed what was recorded)
  cudaEvent_t* ev = nullptr;
  int* kind = nullptr;  // -1 marks the end of a call
  int* pass = nullptr;
};
Timer g_timer;

// Record an event before a launch (kind >= 0) or after a call's last one (-1).
void tick(cudaStream_t s, int kind, int pass) {
  if (!g_timer.on) return;
  std::lock_guard<std::mutex> lk(g_timer.mu);
  if (!g_timer.on) return;
  if (kind >= 0) ++g_timer.launches;
  if (g_timer.used >= g_timer.cap + 64) return;  // the pool has 64 spare end markers
  cudaEventRecord(g_timer.ev[g_timer.used], s);
  g_timer.kind[g_timer.used] = kind;
  g_timer.pass[g_timer.used] = pass;
  ++g_timer.used;
}

// Tracing: an NVTX range around each entry point and each pass's launches
// (host side, header-only NVTX; a no-op unless a profiler is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  NvtxRange(const char* fmt, long long a, long long b) {
    char buf[96];
    std::snprintf(buf, sizeof(buf), fmt, a, b);
    nvtxRangePushA(buf);
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

bool overlaps(const void* a, size_t abytes, const void* b, size_t bbytes) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + bbytes && pb < pa + abytes;
}

}  // namespace

// Test and tuning hooks (scqr3_debug_set): the hand-off wait limit of the
// tensor-core kernels, and whether the tensor-core substitution runs fused.
constexpr long long kDefaultWaitNs = 2000000000ll;
std::atomic<long long> g_wait_ns{kDefaultWaitNs};
std::atomic<int> g_wait_scope{3};  // bit 0: the Gram kernel, bit 1: the substitution kernels
std::atomic<int> g_fused_solve{1};

void set_options(Params* P, const scqr3_opts* opts) {
  const long long w = g_wait_ns.load();
  const int scope = g_wait_scope.load();
  P->wait_ns = (scope & 2) ? w : kDefaultWaitNs;
  P->wait_ns_gram = (scope & 1) ? w : kDefaultWaitNs;
  const double u = 1.1102230246251565e-16;
  P->shift_scale = (opts && opts->shift_scale > 0.0) ? opts->shift_scale : 0.0;
  P->algorithm = (opts && opts->algorithm == SCQR3_ALG_ADAPTIVE) ? 2 : 3;
  // default Alg. 2 tolerance: the bound 6 {mn + n(n+1)} u of Thm. (maincholqr3)
  // (volatile: every product rounded on its own, never contracted into an FMA)
  const double dm = (double)P->m, dn = (double)P->n;
  const volatile double mn = dm * dn, nn1 = dn * (double)(P->n + 1);
  const volatile double sum = mn + nn1;
  const double dflt = 6.0 * sum * u;
  P->tol = (opts && opts->tol > 0.0) ? opts->tol : dflt;
}

}  // namespace scqr3

using namespace scqr3;

extern "C" int scqr3_workspace_bytes(int64_t m, int n, const scqr3_B* B, const scqr3_opts* opts,
                                     size_t* bytes) {
  if (!bytes) return -5;
  const int a = check_args(m, n, B, opts);
  if (a != SCQR3_OK) return a;
  Layout L;
  int grid;
  PassGeom geo;
  const int r = make_layout(m, n, B, opts ? opts->precision : SCQR3_PREC_FP64, 0, &L, &grid, &geo);
  if (r != SCQR3_OK) return r;
  *bytes = L.total;
  return SCQR3_OK;
}

extern "C" int scqr3_host_workspace_bytes(int64_t m, int n, const scqr3_B* B, const scqr3_opts* opts,
                                          size_t* bytes) {
  if (!bytes) return -5;
  const int a = check_args(m, n, B, opts);
  if (a != SCQR3_OK) return a;
  Layout L;
  int grid;
  PassGeom geo;
  const int r = make_layout(m, n, B, opts ? opts->precision : SCQR3_PREC_FP64, 1, &L, &grid, &geo);
  if (r != SCQR3_OK) return r;
  *bytes = L.total;
  return SCQR3_OK;
}

namespace {

// One factorization's launch context: sizes, options, workspace carve-up.
struct Call {
  Params P;
  Layout L;
  int grid = 0;  // pass kernel CTAs (FP64 or mixed)
  PassGeom geo;
  bool mixed = false, csr = false, tc = false;
  bool fused = false;  // tensor-core substitution in one sweep (tc_fused.cu)
  const scqr3_B* B = nullptr;
  cudaStream_t s = nullptr;
  DevState* st = nullptr;
  double *gram = nullptr, *rstack = nullptr, *racc = nullptr, *lt = nullptr, *partials = nullptr;
  double *S = nullptr, *Ra = nullptr;  // n = 256: Cholesky work buffers
  unsigned long long* colmax = nullptr;  // tensor-core Gram: column scales
  double* tcr = nullptr;                 // tensor-core substitution: diagonal blocks of R_k, packed
  double *R = nullptr, *Rpass = nullptr;
  scqr3_info* info = nullptr;
};

// Carves the workspace, fills Params, and queues the state reset and the
// preparation of B. Arguments were checked by the caller.
int setup_call(int64_t m, int n, const scqr3_B* B, const scqr3_opts* opts, void* workspace,
               size_t workspace_bytes, int host_chunks, double* R, double* Rpass, scqr3_info* info,
               cudaStream_t s, Call* c);

// Carves the workspace, fills Params, and queues the state reset and the
// preparation of B. Arguments were checked by the caller.
int begin_call(int64_t m, int n, const scqr3_B* B, const scqr3_opts* opts, void* workspace,
               size_t workspace_bytes, int host_chunks, double* R, double* Rpass, scqr3_info* info,
               cudaStream_t s, Call* c) {
  const int r = setup_call(m, n, B, opts, workspace, workspace_bytes, host_chunks, R, Rpass, info, s, c);
  if (r != SCQR3_OK) return r;
  if (cudaMemsetAsync(c->st, 0, sizeof(DevState), s) != cudaSuccess) return SCQR3_E_CUDA;
  if (cudaMemsetAsync(info, 0, sizeof(scqr3_info), s) != cudaSuccess) return SCQR3_E_CUDA;
  if (B && B->bs > 0) {
    tick(s, SCQR3_KERNEL_BFACTOR, 0);
    launch_bfactor(s, B->bs, B->blocks, m / B->bs, c->lt, c->st, sm_count());
  }
  if (c->csr) {
    tick(s, SCQR3_KERNEL_BFACTOR, 0);
    launch_csr_check(sm_count() * 4, s, m, B, c->st);
  }
  return SCQR3_OK;
}

// The launch context of a call on an existing workspace, without queueing
// anything (a continuing row-partitioned factorization keeps its state).
int setup_call(int64_t m, int n, const scqr3_B* B, const scqr3_opts* opts, void* workspace,
               size_t workspace_bytes, int host_chunks, double* R, double* Rpass, scqr3_info* info,
               cudaStream_t s, Call* c) {
  if (((uintptr_t)workspace & 255) != 0) return SCQR3_E_WORKSPACE;
  c->mixed = opts && (opts->precision == SCQR3_PREC_MIXED || opts->precision == SCQR3_PREC_MIXED_TC);
  c->tc = opts && (opts->precision == SCQR3_PREC_TC || opts->precision == SCQR3_PREC_MIXED_TC);
  const int r = make_layout(m, n, B, opts ? opts->precision : SCQR3_PREC_FP64, host_chunks, &c->L, &c->grid,
                            &c->geo);
  if (r != SCQR3_OK) return r;
  if (workspace_bytes < c->L.total) return SCQR3_E_WORKSPACE;
  char* ws = (char*)workspace;
  c->B = B;
  c->s = s;
  c->csr = B && B->bs == 0;
  c->st = (DevState*)(ws + c->L.state);
  c->gram = (double*)(ws + c->L.gram);
  c->rstack = (double*)(ws + c->L.rstack);
  c->racc = (double*)(ws + c->L.racc);
  c->lt = (B && B->bs > 0) ? (double*)(ws + c->L.lt) : nullptr;
  c->partials = (double*)(ws + c->L.partials);
  c->S = (double*)(ws + c->L.chol);
  c->colmax = (unsigned long long*)(ws + c->L.colmax);
  c->tcr = (double*)(ws + c->L.tcr);
  c->Ra = c->S + pk_size(256);
  c->R = R;
  c->Rpass = Rpass;
  c->info = info;

  Params& P = c->P;
  P.m = m;
  P.n = n;
  P.np = c->tc ? tc_np(n) : padded_n(n);
  P.max_passes = (opts && opts->max_passes) ? opts->max_passes : 6;
  P.bs = B ? B->bs : 0;
  P.norm_x2 = opts ? opts->norm_x2 : 0.0;
  P.normb_in = B ? B->norm2 : 0.0;
  P.csr = c->csr ? 1 : 0;
  P.tc = c->tc ? 1 : 0;
  P.solve_only = (c->csr || c->tc) ? 1 : 0;
  set_options(&P, opts);
  c->fused = c->tc && !c->mixed && g_fused_solve.load() != 0 && tc_fused_supported(n);
  return SCQR3_OK;
}

// The first Gram matrix (of X) over rows [r0, r1), into the partial slots
// from `slot0` on; returns the number of slots written. The whole range
// (0, m) gives exactly the launch of the fixed sequence.
int first_gram(Call& c, const double* X, int64_t ldx, int64_t r0, int64_t r1, int slot0) {
  Params Pc = c.P;
  Pc.m = r1 - r0;
  const double* src = X + r0 * ldx;
  double* part = c.partials + (int64_t)slot0 * c.L.part_stride;
  tick(c.s, SCQR3_KERNEL_GRAM, 0);
  if (c.tc) {
    const int g = tc_grid(Pc.m, c.P.np, sm_count());
    launch_tc_gram(g, sm_count(), c.s, src, ldx, Pc, -1, c.colmax, part, c.L.part_stride, c.st, 0, c.lt,
                   c.lt ? r0 / c.P.bs : 0, 1, 0);
    return g;
  }
  if (c.P.np == 256) {
    launch_gram256(c.grid, c.s, src, ldx, Pc, -1, part, c.L.part_stride, c.st);
    return c.grid;
  }
  if (c.csr) {  // the whole matrix only: rows reach across any split
    launch_csr_gram(c.P.np, c.L.csr_grid, c.s, src, ldx, c.P, -1, c.B, part, c.L.part_stride, c.st);
    return c.L.n_partials;
  }
  if (c.mixed) {
    const int64_t pn = (Pc.m + df_rows_per_panel(c.P.np) - 1) / df_rows_per_panel(c.P.np);
    const int g = (int)(pn < c.grid ? (pn < 1 ? 1 : pn) : c.grid);
    launch_df_pass(c.P.np, g, c.s, src, ldx, nullptr, 0, Pc, -1, nullptr, part, c.L.part_stride, c.st);
    return g * df_groups(c.P.np);
  }
  const int64_t pn = (Pc.m + c.geo.pr - 1) / c.geo.pr;
  const int g = (int)(pn < c.grid ? (pn < 1 ? 1 : pn) : c.grid);
  launch_pass(c.P.np, g, c.s, src, ldx, nullptr, 0, Pc, -1, nullptr, c.lt, part, c.L.part_stride, c.st);
  return g * c.geo.groups;
}

void launch_any_chol(Call& c, int pass) {
  tick(c.s, SCQR3_KERNEL_CHOL, pass);
  if (c.P.np == 256)
    launch_chol256(c.s, c.P, pass, c.gram, c.rstack, c.racc, c.R, c.Rpass, c.st, c.info, c.S, c.Ra);
  else
    launch_chol(c.P.np, c.s, c.P, pass, c.gram, c.rstack, c.racc, c.R, c.Rpass, c.st, c.info);
}

// Pass k's solve Q := Q R_k^{-1} over rows [r0, r1) (src -> dst), with the
// fused Gram when the device asks for it (FP64 and mixed forms, whole range
// only: a range is used only for a final solve, which has no Gram).
// CTAs of the pass kernel for a padded size and m rows.
int pass_grid(int np, int64_t m) {
  int gm = 0;
  PassGeom geo;
  if (device_geo(np, &gm, &geo) != cudaSuccess) return 1;
  const int64_t pn = (m + geo.pr - 1) / geo.pr;
  return (int)(pn < gm ? (pn < 1 ? 1 : pn) : gm);
}

// Width of the diagonal blocks of the tensor-core substitution: 16 columns
// halve the FP64 work again but multiply the tensor-core updates.
int tc_block_width(int n) { return n <= 64 ? 16 : 32; }

// The tensor-core form's substitution (n <= 256) in blocks of w columns: for
// J = 0, 1, ..: Y_J = X_J R_JJ^{-1} (FP64 pass kernel), then X_K := X_K -
// Y_J R_JK for the later columns, 32 at a time (tensor cores, exact digit
// split). Block 0 reads the pass's input; every later block is updated and
// solved in place in the output.
// The fused substitution (tc_fused.cu: one sweep, column maxima of the result
// for the next Gram matrix) serves the FP64-accurate tensor-core form for
// 16 < n <= 64.
bool use_fused(const Call& c) { return c.fused; }

void tc_solve_rows(Call& c, int k, const double* rk, const double* src, int64_t lds, double* dst, int64_t ldd,
                   const Params& Pc) {
  if (use_fused(c)) {
    // B = I: the column maxima go to the next Gram matrix (the oblique one
    // scans Z = L^T Q itself)
    unsigned long long* cm = c.lt ? nullptr : c.colmax;
    if (cm) cudaMemsetAsync(cm, 0, sizeof(unsigned long long) * 256, c.s);
    tick(c.s, SCQR3_KERNEL_PASS, k);
    launch_tc_fused(sm_count(), c.s, src, lds, dst, ldd, Pc, k, rk, cm, c.st);
    return;
  }
  const int n = Pc.n, w = tc_block_width(n), nb = (n + w - 1) / w;
  tick(c.s, SCQR3_KERNEL_TCUPDATE, k);
  launch_tc_split_r(c.s, rk, c.P.np, n, w, k, c.st, c.tcr);
  for (int J = 0; J < nb; ++J) {
    const int wj = n - w * J < w ? n - w * J : w;
    const int npj = wj <= 16 ? 16 : 32;
    Params PJ = Pc;
    PJ.n = wj;
    PJ.np = npj;
    tick(c.s, SCQR3_KERNEL_PASS, k);
    const double* in = J == 0 ? src : dst + w * J;
    const int64_t ldin = J == 0 ? lds : ldd;
    launch_pass(npj, pass_grid(npj, Pc.m), c.s, in, ldin, dst + w * J, ldd, PJ, k, c.tcr + J * pk_size(32),
                nullptr, c.partials, c.L.part_stride, c.st);
    for (int c0 = w * (J + 1); c0 < n; c0 += 32) {
      const int n1 = n - c0 < 32 ? n - c0 : 32;
      tick(c.s, SCQR3_KERNEL_TCUPDATE, k);
      const double* x1 = J == 0 ? src + c0 : dst + c0;
      const int64_t ldx1 = J == 0 ? lds : ldd;
      launch_tc_update(sm_count(), c.s, w, dst + w * J, ldd, x1, ldx1, dst + c0, ldd, Pc.m, n1, k, rk, c.P.np,
                       w * J, c0, 0, w, c.st, c.P.wait_ns);
    }
  }
}

void solve_rows(Call& c, int k, const double* src, int64_t lds, double* dst, int64_t ldd, int64_t r0,
                int64_t r1) {
  Params Pc = c.P;
  Pc.m = r1 - r0;
  src += r0 * lds;
  dst += r0 * ldd;
  const double* rk = c.rstack + (size_t)k * pk_size(c.P.np);
  if (c.tc && !c.mixed) {
    tc_solve_rows(c, k, rk, src, lds, dst, ldd, Pc);
    return;
  }
  if (c.P.np == 256) {
    tick(c.s, SCQR3_KERNEL_TRSM, k);
    launch_trsm256(trsm256_grid(Pc.m), c.s, src, lds, dst, ldd, Pc, k, rk, c.st);
    return;
  }
  tick(c.s, SCQR3_KERNEL_PASS, k);
  if (c.mixed) {
    const int64_t pn = (Pc.m + df_rows_per_panel(c.P.np) - 1) / df_rows_per_panel(c.P.np);
    const int g = (int)(pn < c.grid ? (pn < 1 ? 1 : pn) : c.grid);
    launch_df_pass(c.P.np, g, c.s, src, lds, dst, ldd, Pc, k, rk, c.partials, c.L.part_stride, c.st);
  } else {
    const int64_t pn = (Pc.m + c.geo.pr - 1) / c.geo.pr;
    const int g = (int)(pn < c.grid ? (pn < 1 ? 1 : pn) : c.grid);
    launch_pass(c.P.np, g, c.s, src, lds, dst, ldd, Pc, k, rk, c.lt, c.partials, c.L.part_stride, c.st);
  }
}

// After pass k: the separate Gram kernels (n = 256, tensor cores, CSR B) and
// the fixed-order sum of the partial Gram matrices into `out`.
void after_pass_gram(Call& c, int k, const double* Q, int64_t ldq, double* out);

// After pass k: the next Gram matrix and the Cholesky of pass k + 1.
void after_pass(Call& c, int k, const double* Q, int64_t ldq) {
  after_pass_gram(c, k, Q, ldq, c.gram);
  launch_any_chol(c, k + 1);
}

void after_pass_gram(Call& c, int k, const double* Q, int64_t ldq, double* out) {
  if (c.tc) {
    tick(c.s, SCQR3_KERNEL_GRAM, k + 1);
    // the mixed form keeps float pairs between passes
    launch_tc_gram(c.L.tc_grid, sm_count(), c.s, Q, ldq, c.P, k, c.colmax, c.partials, c.L.part_stride, c.st,
                   c.mixed ? 1 : 0, c.lt, 0, (use_fused(c) && !c.lt) ? 0 : 1, 0);
  } else if (c.P.np == 256) {
    tick(c.s, SCQR3_KERNEL_GRAM, k + 1);
    launch_gram256(c.grid, c.s, Q, ldq, c.P, k, c.partials, c.L.part_stride, c.st);
  } else if (c.csr) {
    tick(c.s, SCQR3_KERNEL_GRAM, k + 1);
    launch_csr_gram(c.P.np, c.L.csr_grid, c.s, Q, ldq, c.P, k, c.B, c.partials, c.L.part_stride, c.st);
  }
  tick(c.s, SCQR3_KERNEL_REDUCE, k + 1);
  launch_reduce(c.s, c.partials, c.L.n_partials, c.L.part_stride, out, c.st, k);
}

int check_factor_pointers(const double* X, int64_t m, int n, int64_t ldx, const double* Q, int64_t ldq,
                          const double* R, const void* workspace, const void* info) {
  if (!X) return -1;
  if (ldx < n) return -4;
  if (!Q) return -6;
  if (ldq < n) return -7;
  if (!R) return -8;
  if (!workspace) return -10;
  if (!info) return -13;
  // Q may be X itself (in place) but must not overlap it otherwise.
  const size_t xbytes = sizeof(double) * (size_t)((m - 1) * ldx + n);
  const size_t qbytes = sizeof(double) * (size_t)((m - 1) * ldq + n);
  if ((const void*)Q != (const void*)X && overlaps(X, xbytes, Q, qbytes)) return -6;
  if ((const void*)Q == (const void*)X && ldq != ldx) return -7;
  return SCQR3_OK;
}

}  // namespace

namespace scqr3 {

// For the tensor-core adjoint (adjoint.cu), which runs the factorization's
// kernels: their attributes set on the current device (once), its SM count,
// the pass kernel's grid for m rows, and whether the one-sweep substitution
// serves n columns.
int tc_kernels_ready(int* sms) {
  int gm = 0;
  PassGeom geo;
  if (device_geo(64, &gm, &geo) != cudaSuccess) return SCQR3_E_CUDA;
  *sms = sm_count();
  return SCQR3_OK;
}
int pass_kernel_grid(int np, int64_t m) { return pass_grid(np, m); }
bool fused_solve_selected(int n) { return g_fused_solve.load() != 0 && tc_fused_supported(n); }

}  // namespace scqr3

extern "C" int scqr3_factor(const double* X, int64_t m, int n, int64_t ldx, const scqr3_B* B,
                            double* Q, int64_t ldq, double* R, double* Rpass, void* workspace,
                            size_t workspace_bytes, const scqr3_opts* opts, scqr3_info* info,
                            void* stream) {
  int a = check_args(m, n, B, opts);
  if (a != SCQR3_OK) return a;
  a = check_factor_pointers(X, m, n, ldx, Q, ldq, R, workspace, info);
  if (a != SCQR3_OK) return a;
  NvtxRange range("scqr3_factor %lld x %lld", (long long)m, (long long)n);
  Call c;
  a = begin_call(m, n, B, opts, workspace, workspace_bytes, 0, R, Rpass, info, (cudaStream_t)stream, &c);
  if (a != SCQR3_OK) return a;

  // Pass 1 of Alg. 3: A = X^T X (or X^T B X), then the fixed sequence of
  // passes whose launches the device skips once they are not needed.
  {
    NvtxRange g("scqr3 first Gram");
    const int slots = first_gram(c, X, ldx, 0, m, 0);
    tick(c.s, SCQR3_KERNEL_REDUCE, 0);
    launch_reduce(c.s, c.partials, slots, c.L.part_stride, c.gram, c.st, -1);
    launch_any_chol(c, 0);
  }
  for (int k = 0; k < c.P.max_passes; ++k) {
    NvtxRange pr("scqr3 pass %lld of %lld", (long long)k, (long long)c.P.max_passes);
    solve_rows(c, k, k == 0 ? X : Q, k == 0 ? ldx : ldq, Q, ldq, 0, m);
    if (k + 1 < c.P.max_passes) after_pass(c, k, Q, ldq);
  }
  if (c.mixed) {  // float pairs remain when the last solve was followed by a Gram step
    tick(c.s, SCQR3_KERNEL_FINISH, -1);
    launch_df_finish(sm_count() * 4, c.s, Q, ldq, m, n, c.P.max_passes, c.st);
  }
  // a tensor-core kernel after the last Cholesky may have recorded a failure
  if (c.tc) launch_status(c.s, c.st, c.info);
  tick(c.s, -1, -1);
  if (cudaGetLastError() != cudaSuccess) return SCQR3_E_CUDA;
  return SCQR3_OK;
}

namespace {
// A copy stream, chunk events and a pinned staging slot for the pass flags,
// per device; a call holds the device's lock while it runs.
struct HostRes {
  bool ready = false;
  cudaStream_t copy = nullptr;
  cudaEvent_t entry = nullptr;
  cudaEvent_t up[kHostChunks], down[kHostChunks];
  DevState* flags = nullptr;  // pinned host memory
  std::mutex mu;
};
HostRes g_host[kMaxDevices];

int host_res(HostRes** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SCQR3_E_CUDA;
  HostRes& h = g_host[dev];
  std::lock_guard<std::mutex> lk(g_mu);
  if (!h.ready) {
    if (cudaStreamCreateWithFlags(&h.copy, cudaStreamNonBlocking) != cudaSuccess) return SCQR3_E_CUDA;
    if (cudaEventCreateWithFlags(&h.entry, cudaEventDisableTiming) != cudaSuccess) return SCQR3_E_CUDA;
    for (int i = 0; i < kHostChunks; ++i) {
      if (cudaEventCreateWithFlags(&h.up[i], cudaEventDisableTiming) != cudaSuccess) return SCQR3_E_CUDA;
      if (cudaEventCreateWithFlags(&h.down[i], cudaEventDisableTiming) != cudaSuccess) return SCQR3_E_CUDA;
    }
    if (cudaMallocHost((void**)&h.flags, sizeof(DevState)) != cudaSuccess) return SCQR3_E_CUDA;
    h.ready = true;
  }
  *out = &h;
  return SCQR3_OK;
}
}  // namespace

extern "C" int scqr3_factor_host(const double* X, int64_t m, int n, int64_t ldx, const scqr3_B* B,
                                 double* Q, int64_t ldq, double* R, double* Qdev, void* workspace,
                                 size_t workspace_bytes, const scqr3_opts* opts, scqr3_info* info,
                                 void* stream) {
  int a = check_args(m, n, B, opts);
  if (a != SCQR3_OK) return a;
  a = check_factor_pointers(X, m, n, ldx, Q, ldq, R, workspace, info);
  if (a != SCQR3_OK) return a;
  if (!Qdev) return -9;
  HostRes* h = nullptr;
  a = host_res(&h);
  if (a != SCQR3_OK) return a;
  std::lock_guard<std::mutex> lk(h->mu);
  NvtxRange range("scqr3_factor_host %lld x %lld", (long long)m, (long long)n);
  cudaStream_t s = (cudaStream_t)stream;
  Call c;
  {
    // R and info live in the workspace until the end of the call
    Layout L;
    int grid;
    PassGeom geo;
    a = make_layout(m, n, B, opts ? opts->precision : SCQR3_PREC_FP64, 1, &L, &grid, &geo);
    if (a != SCQR3_OK) return a;
    if (workspace_bytes < L.total || ((uintptr_t)workspace & 255) != 0) return SCQR3_E_WORKSPACE;
    char* ws = (char*)workspace;
    a = begin_call(m, n, B, opts, workspace, workspace_bytes, 1, (double*)(ws + L.rdev), nullptr,
                   (scqr3_info*)(ws + L.infodev), s, &c);
    if (a != SCQR3_OK) return a;
  }
  const size_t row_bytes = sizeof(double) * (size_t)n;
  const int64_t cr = host_chunk_rows(m);
  const int nchunks = (int)((m + cr - 1) / cr);

  // X -> Qdev in chunks on the copy stream (after the caller's earlier work on
  // `stream`); with B = I each chunk's share of the first Gram starts as soon
  // as it has arrived.
  if (cudaEventRecord(h->entry, s) != cudaSuccess) return SCQR3_E_CUDA;
  if (cudaStreamWaitEvent(h->copy, h->entry, 0) != cudaSuccess) return SCQR3_E_CUDA;
  int slots = 0;
  for (int ci = 0; ci < nchunks; ++ci) {
    const int64_t r0 = ci * cr, r1 = (r0 + cr) < m ? (r0 + cr) : m;
    if (cudaMemcpy2DAsync(Qdev + r0 * n, row_bytes, X + r0 * ldx, sizeof(double) * ldx, row_bytes,
                          (size_t)(r1 - r0), cudaMemcpyHostToDevice, h->copy) != cudaSuccess)
      return SCQR3_E_CUDA;
    if (cudaEventRecord(h->up[ci], h->copy) != cudaSuccess) return SCQR3_E_CUDA;
    if (!B) {
      if (cudaStreamWaitEvent(s, h->up[ci], 0) != cudaSuccess) return SCQR3_E_CUDA;
      slots += first_gram(c, Qdev, n, r0, r1, slots);
    }
  }
  if (B) {
    if (cudaStreamWaitEvent(s, h->up[nchunks - 1], 0) != cudaSuccess) return SCQR3_E_CUDA;
    slots = first_gram(c, Qdev, n, 0, m, 0);
  }
  tick(s, SCQR3_KERNEL_REDUCE, 0);
  launch_reduce(s, c.partials, slots, c.L.part_stride, c.gram, c.st, -1);
  launch_any_chol(c, 0);

  // Passes, driven from the host: after each Cholesky the device's flags say
  // whether pass k solves and whether a Gram follows. The last solve runs in
  // row chunks whose copies back to Q overlap the next chunk's solve.
  bool copied = false;
  for (int k = 0; k < c.P.max_passes; ++k) {
    if (cudaMemcpyAsync(h->flags, c.st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return SCQR3_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SCQR3_E_CUDA;
    if (!h->flags->run_trsm[k]) break;
    if (h->flags->gram_after[k]) {
      solve_rows(c, k, Qdev, n, Qdev, n, 0, m);
      if (k + 1 < c.P.max_passes) after_pass(c, k, Qdev, n);
      continue;
    }
    for (int ci = 0; ci < nchunks; ++ci) {
      const int64_t r0 = ci * cr, r1 = (r0 + cr) < m ? (r0 + cr) : m;
      solve_rows(c, k, Qdev, n, Qdev, n, r0, r1);
      if (cudaEventRecord(h->down[ci], s) != cudaSuccess) return SCQR3_E_CUDA;
      if (cudaStreamWaitEvent(h->copy, h->down[ci], 0) != cudaSuccess) return SCQR3_E_CUDA;
      if (cudaMemcpy2DAsync(Q + r0 * ldq, sizeof(double) * ldq, Qdev + r0 * n, row_bytes, row_bytes,
                            (size_t)(r1 - r0), cudaMemcpyDeviceToHost, h->copy) != cudaSuccess)
        return SCQR3_E_CUDA;
    }
    copied = true;
    break;
  }
  if (!copied) {  // stopped by Alg. 2's test or a failure: Q as the device left it
    if (c.mixed) {
      tick(s, SCQR3_KERNEL_FINISH, -1);
      launch_df_finish(sm_count() * 4, s, Qdev, n, m, n, c.P.max_passes, c.st);
    }
    if (cudaEventRecord(h->down[0], s) != cudaSuccess) return SCQR3_E_CUDA;
    if (cudaStreamWaitEvent(h->copy, h->down[0], 0) != cudaSuccess) return SCQR3_E_CUDA;
    if (cudaMemcpy2DAsync(Q, sizeof(double) * ldq, Qdev, row_bytes, row_bytes, (size_t)m,
                          cudaMemcpyDeviceToHost, h->copy) != cudaSuccess)
      return SCQR3_E_CUDA;
  }
  if (c.tc) launch_status(s, c.st, c.info);
  tick(s, -1, -1);
  if (cudaMemcpyAsync(R, c.R, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return SCQR3_E_CUDA;
  if (cudaMemcpyAsync(info, c.info, sizeof(scqr3_info), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return SCQR3_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SCQR3_E_CUDA;
  if (cudaStreamSynchronize(h->copy) != cudaSuccess) return SCQR3_E_CUDA;
  if (cudaGetLastError() != cudaSuccess) return SCQR3_E_CUDA;
  return SCQR3_OK;
}

// ---- row-partitioned form ------------------------------------------------------------------

namespace {
// The forms the row-partitioned calls take (see include/scqr3.h); codes in
// scqr3_factor's numbering.
int check_shard(int64_t m_local, int n, const scqr3_B* B, const scqr3_opts* opts) {
  const int a = check_args(m_local, n, B, opts, true);
  if (a != SCQR3_OK) return a;
  if (opts && (opts->precision == SCQR3_PREC_MIXED || opts->precision == SCQR3_PREC_MIXED_TC))
    return SCQR3_E_UNSUPPORTED;
  if (B && B->bs == 0) return SCQR3_E_UNSUPPORTED;
  if (B && !(B->norm2 > 0.0)) return -5;
  return SCQR3_OK;
}

// scqr3_factor's argument codes (m -2, n -3, B -5, opts -12) in another
// prototype's positions.
int remap(int r, int m_pos, int n_pos, int b_pos, int o_pos) {
  switch (r) {
    case -2: return -m_pos;
    case -3: return -n_pos;
    case -5: return -b_pos;
    case -12: return -o_pos;
    default: return r;
  }
}
}  // namespace

extern "C" int scqr3_shard_sizes(int64_t m_local, int n, const scqr3_B* B, const scqr3_opts* opts,
                                 size_t* workspace_bytes, size_t* gram_words) {
  if (!workspace_bytes) return -5;
  if (!gram_words) return -6;
  const int a = check_shard(m_local, n, B, opts);
  if (a != SCQR3_OK) return remap(a, 1, 2, 3, 4);
  Layout L;
  int grid;
  PassGeom geo;
  const int prec = opts ? opts->precision : SCQR3_PREC_FP64;
  const int r = make_layout(m_local, n, B, prec, 0, &L, &grid, &geo);
  if (r != SCQR3_OK) return r;
  *workspace_bytes = L.total;
  *gram_words = (size_t)L.part_stride;
  return SCQR3_OK;
}

extern "C" int scqr3_gram_partial(const double* X, int64_t m_local, int n, int64_t ldx, const scqr3_B* B,
                                  double* G, void* workspace, size_t workspace_bytes, const scqr3_opts* opts,
                                  scqr3_info* info, void* stream) {
  int a = check_shard(m_local, n, B, opts);
  if (a != SCQR3_OK) return remap(a, 2, 3, 5, 9);
  if (!X) return -1;
  if (ldx < n) return -4;
  if (!G) return -6;
  if (!workspace) return -7;
  if (!info) return -10;
  NvtxRange range("scqr3_gram_partial %lld x %lld", (long long)m_local, (long long)n);
  Call c;
  a = begin_call(m_local, n, B, opts, workspace, workspace_bytes, 0, nullptr, nullptr, info, (cudaStream_t)stream,
                 &c);
  if (a != SCQR3_OK) return a;
  const int slots = first_gram(c, X, ldx, 0, m_local, 0);
  tick(c.s, SCQR3_KERNEL_REDUCE, 0);
  launch_reduce(c.s, c.partials, slots, c.L.part_stride, G, c.st, -1);
  tick(c.s, -1, -1);
  if (cudaGetLastError() != cudaSuccess) return SCQR3_E_CUDA;
  return SCQR3_OK;
}

extern "C" int scqr3_apply_pass(int pass, const double* G, int64_t m_global, const double* X, int64_t m_local,
                                int n, int64_t ldx, const scqr3_B* B, double* Q, int64_t ldq, double* R,
                                double* G_next, void* workspace, size_t workspace_bytes, const scqr3_opts* opts,
                                scqr3_info* info, void* stream) {
  int a = check_shard(m_local, n, B, opts);
  if (a != SCQR3_OK) return remap(a, 5, 6, 8, 15);
  const int max_passes = (opts && opts->max_passes) ? opts->max_passes : 6;
  if (pass < 0 || pass >= max_passes) return -1;
  if (!G) return -2;
  if (m_global < n || m_global < m_local) return -3;
  if (!X) return -4;
  if (ldx < n) return -7;
  if (!Q) return -9;
  if (ldq < n) return -10;
  if (!R) return -11;
  if (!G_next && pass + 1 < max_passes) return -12;
  if (!workspace) return -13;
  if (!info) return -16;
  const size_t xbytes = sizeof(double) * (size_t)((m_local - 1) * ldx + n);
  const size_t qbytes = sizeof(double) * (size_t)((m_local - 1) * ldq + n);
  if ((const void*)Q != (const void*)X && overlaps(X, xbytes, Q, qbytes)) return -9;
  if ((const void*)Q == (const void*)X && ldq != ldx) return -10;
  NvtxRange range("scqr3_apply_pass %lld, %lld rows", (long long)pass, (long long)m_local);
  Call c;
  a = setup_call(m_local, n, B, opts, workspace, workspace_bytes, 0, R, nullptr, info, (cudaStream_t)stream, &c);
  if (a != SCQR3_OK) return a;
  // the shift, Alg. 2's tolerance and the pass decisions are those of the
  // whole X: the Cholesky kernel sees the global m
  Params Pg = c.P;
  Pg.m = m_global;
  set_options(&Pg, opts);
  tick(c.s, SCQR3_KERNEL_CHOL, pass);
  if (c.P.np == 256)
    launch_chol256(c.s, Pg, pass, G, c.rstack, c.racc, c.R, nullptr, c.st, c.info, c.S, c.Ra);
  else
    launch_chol(c.P.np, c.s, Pg, pass, G, c.rstack, c.racc, c.R, nullptr, c.st, c.info);
  solve_rows(c, pass, pass == 0 ? X : Q, pass == 0 ? ldx : ldq, Q, ldq, 0, m_local);
  if (pass + 1 < max_passes) after_pass_gram(c, pass, Q, ldq, G_next);
  if (c.tc) launch_status(c.s, c.st, c.info);
  tick(c.s, -1, -1);
  if (cudaGetLastError() != cudaSuccess) return SCQR3_E_CUDA;
  return SCQR3_OK;
}

extern "C" int scqr3_debug_set(int key, long long value) {
  switch (key) {
    case SCQR3_DEBUG_WAIT_NS:
      g_wait_ns.store(value < 0 ? kDefaultWaitNs : value);
      return SCQR3_OK;
    case SCQR3_DEBUG_WAIT_SCOPE:
      if (value < 0 || value > 3) return -2;
      g_wait_scope.store((int)value);
      return SCQR3_OK;
    case SCQR3_DEBUG_FUSED_SOLVE:
      if (value != 0 && value != 1) return -2;
      g_fused_solve.store((int)value);
      return SCQR3_OK;
    default:
      return -1;
  }
}

extern "C" int scqr3_timing_begin(int capacity) {
  if (capacity < 1) return -1;
  std::lock_guard<std::mutex> lk(g_timer.mu);
  if (g_timer.ev) {
    for (int i = 0; i < g_timer.cap + 64; ++i) cudaEventDestroy(g_timer.ev[i]);
    delete[] g_timer.ev;
    delete[] g_timer.kind;
    delete[] g_timer.pass;
    g_timer.ev = nullptr;
  }
  g_timer.cap = capacity;
  g_timer.ev = new cudaEvent_t[capacity + 64];
  g_timer.kind = new int[capacity + 64];
  g_timer.pass = new int[capacity + 64];
  for (int i = 0; i < capacity + 64; ++i)
    if (cudaEventCreate(&g_timer.ev[i]) != cudaSuccess) return SCQR3_E_CUDA;
  g_timer.used = 0;
  g_timer.launches = 0;
  g_timer.on = true;
  return SCQR3_OK;
}

extern "C" int scqr3_timing_end(scqr3_launch_time* out, int capacity, int* count) {
  std::lock_guard<std::mutex> lk(g_timer.mu);
  g_timer.on = false;
  if (count) *count = g_timer.launches;
  if (!g_timer.ev) return SCQR3_OK;
  if (g_timer.used > 0 && cudaEventSynchronize(g_timer.ev[g_timer.used - 1]) != cudaSuccess)
    return SCQR3_E_CUDA;
  int k = 0;
  for (int i = 0; i + 1 < g_timer.used && k < capacity; ++i) {
    if (g_timer.kind[i] < 0) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g_timer.ev[i], g_timer.ev[i + 1]) != cudaSuccess) return SCQR3_E_CUDA;
    if (out) {
      out[k].kernel = g_timer.kind[i];
      out[k].pass = g_timer.pass[i];
      out[k].ms = ms;
    }
    ++k;
  }
  return SCQR3_OK;
}
