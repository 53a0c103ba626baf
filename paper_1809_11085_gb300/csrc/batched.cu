// batched.cu -- many independent, uneven tall-skinny factorizations in one
// fixed launch sequence (FP64, B = I).
//
// Each phase is ONE persistent launch over the whole batch: CTAs (one per
// SM) take tiles -- a run of row panels of one matrix -- from an atomic
// queue, largest size class first, and run that matrix's pass on them (the
// same pass_segment code as the single-matrix kernel, instantiated for each
// padded size). A matrix that needs no work in this pass (finished, failed,
// or not needing a Gram) makes its tiles return at once, so matrices that
// need an extra shifted pass (Alg. 2) cost only their own tiles. Every tile
// writes its partial Gram matrix to a slot of its own; the per-matrix
// reduction then sums the matrix's tiles in tile order, so the result does
// not depend on which CTA ran which tile. The per-matrix shift, Cholesky and
// pass bookkeeping run as one launch with one CTA per matrix.
//
// Host side: scqr3_batch_plan_create validates the items and lays out the
// workspace and the tile list (host memory only); scqr3_batch_plan_upload
// copies the tables into the workspace once; scqr3_factor_batched then only
// queues memsets and kernels, so it can be captured in a CUDA graph and
// replayed.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "fp64_device.cuh"

namespace scqr3 {

struct BItem {
  const double* X;
  double* Q;
  double* R;
  double* Rpass;
  scqr3_info* info;
  DevState* st;
  double* gram;
  double* rstack;
  double* racc;
  Params P;
  int64_t ldx, ldq;
  int tile_lo, tile_hi;  // this matrix's tiles in the global tile list
};

struct BTile {
  int item;
  int np;
  int64_t p_begin, p_end;  // row panels [p_begin, p_end)
  int64_t slot;            // offset (doubles) of this tile's partial Gram slot
};

// Shapes of the FP64 pass kernel (rows per panel, Gram groups, shared memory).
int batched_rows_per_panel(int np) {
  return np == 16 ? Geo<16>::PR : np == 32 ? Geo<32>::PR : np == 64 ? Geo<64>::PR : Geo<128>::PR;
}
int batched_groups(int np) {
  return np == 16 ? Geo<16>::G : np == 32 ? Geo<32>::G : np == 64 ? Geo<64>::G : Geo<128>::G;
}
size_t batched_pass_smem() {
  return std::max(std::max(Geo<16>::smem, Geo<32>::smem), std::max(Geo<64>::smem, Geo<128>::smem));
}
size_t batched_chol_smem() { return 2 * sizeof(double) * pk_size(128); }

template <int NP>
__device__ __forceinline__ void run_tile(const BItem& it, const BTile& t, int pass, double* scratch,
                                         double* slots) {
  constexpr int E = pk_size(NP);
  constexpr int G = Geo<NP>::G;
  const double* src = (pass <= 0) ? it.X : it.Q;
  const int64_t lds = (pass <= 0) ? it.ldx : it.ldq;
  const double* rk = pass >= 0 ? it.rstack + (int64_t)pass * E : nullptr;
  pass_segment<NP>(src, lds, it.Q, it.ldq, it.P, pass, rk, nullptr, scratch, E + 1, it.st, t.p_begin,
                   t.p_end, 1);
  __syncthreads();
  // fixed-order sum of the CTA's group slots into this tile's slot
  double* out = slots + t.slot;
  for (int e = threadIdx.x; e <= E; e += blockDim.x) {
    double s = 0.0;
    for (int g2 = 0; g2 < G; ++g2) s += scratch[(int64_t)g2 * (E + 1) + e];
    out[e] = s;
  }
}

__global__ void __launch_bounds__(kThreads, 1)
batched_pass_kernel(const BItem* __restrict__ items, const BTile* __restrict__ tiles, int ntiles, int pass,
                    int* __restrict__ counter, double* __restrict__ scratch_all, int scratch_stride,
                    double* __restrict__ slots) {
  __shared__ int t_sh;
  double* scratch = scratch_all + (int64_t)blockIdx.x * scratch_stride;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) t_sh = atomicAdd(counter, 1);
    __syncthreads();
    const int t = t_sh;
    if (t >= ntiles) break;
    const BTile tile = tiles[t];
    const BItem& it = items[tile.item];
    if (pass >= 0 && !(it.st->run_trsm[pass] && it.st->gram_after[pass])) {
      // solve only (last pass) or nothing: no Gram slot is read for this tile
      if (pass >= 0 && it.st->run_trsm[pass]) {
        switch (tile.np) {
          case 16: pass_segment<16>(it.Q, it.ldq, it.Q, it.ldq, it.P, pass, it.rstack + (int64_t)pass * pk_size(16), nullptr, scratch, pk_size(16) + 1, it.st, tile.p_begin, tile.p_end, 1); break;
          case 32: pass_segment<32>(it.Q, it.ldq, it.Q, it.ldq, it.P, pass, it.rstack + (int64_t)pass * pk_size(32), nullptr, scratch, pk_size(32) + 1, it.st, tile.p_begin, tile.p_end, 1); break;
          case 64: pass_segment<64>(it.Q, it.ldq, it.Q, it.ldq, it.P, pass, it.rstack + (int64_t)pass * pk_size(64), nullptr, scratch, pk_size(64) + 1, it.st, tile.p_begin, tile.p_end, 1); break;
          default: pass_segment<128>(it.Q, it.ldq, it.Q, it.ldq, it.P, pass, it.rstack + (int64_t)pass * pk_size(128), nullptr, scratch, pk_size(128) + 1, it.st, tile.p_begin, tile.p_end, 1); break;
        }
        // pass 0 reads X: handled below (pass 0 always has a Gram after it unless max_passes == 1)
      }
      continue;
    }
    switch (tile.np) {
      case 16: run_tile<16>(it, tile, pass, scratch, slots); break;
      case 32: run_tile<32>(it, tile, pass, scratch, slots); break;
      case 64: run_tile<64>(it, tile, pass, scratch, slots); break;
      default: run_tile<128>(it, tile, pass, scratch, slots); break;
    }
  }
}

// Per-matrix fixed-order sum of its tiles' slots: A = sum over tiles in order.
__global__ void batched_reduce_kernel(const BItem* __restrict__ items, const BTile* __restrict__ tiles,
                                      const double* __restrict__ slots, int pass) {
  const BItem& it = items[blockIdx.x];
  if (pass >= 0 && !it.st->gram_after[pass]) return;
  const int E = pk_size(it.P.np);
  for (int e = threadIdx.x; e <= E; e += blockDim.x) {
    double s = 0.0;
    for (int t = it.tile_lo; t < it.tile_hi; ++t) s += slots[tiles[t].slot + e];
    it.gram[e] = s;
  }
}

__global__ void __launch_bounds__(512, 1)
batched_chol_kernel(const BItem* __restrict__ items, int pass) {
  const BItem& it = items[blockIdx.x];
  if (pass == 0) {  // a fresh record for this call
    int* w = reinterpret_cast<int*>(it.info);
    for (int e = threadIdx.x; e < (int)(sizeof(scqr3_info) / sizeof(int)); e += blockDim.x) w[e] = 0;
    __syncthreads();
  }
  extern __shared__ __align__(16) double sm[];
  switch (it.P.np) {
    case 16: chol_body<16>(it.P, pass, it.gram, it.rstack, it.racc, it.R, it.Rpass, it.st, it.info, sm, sm + pk_size(16)); break;
    case 32: chol_body<32>(it.P, pass, it.gram, it.rstack, it.racc, it.R, it.Rpass, it.st, it.info, sm, sm + pk_size(32)); break;
    case 64: chol_body<64>(it.P, pass, it.gram, it.rstack, it.racc, it.R, it.Rpass, it.st, it.info, sm, sm + pk_size(64)); break;
    default: chol_body<128>(it.P, pass, it.gram, it.rstack, it.racc, it.R, it.Rpass, it.st, it.info, sm, sm + pk_size(128)); break;
  }
}

}  // namespace scqr3

using namespace scqr3;

struct scqr3_batch_plan {
  int count = 0;
  int max_passes = 6;
  scqr3_opts opts{};      // shift_scale, algorithm and tol apply to every matrix
  bool has_opts = false;
  int grid = 0;
  int ntiles = 0;
  int np_max = 16;
  size_t bytes = 0;
  // workspace offsets
  size_t off_items = 0, off_tiles = 0, off_counters = 0, off_states = 0, off_mats = 0, off_scratch = 0,
         off_slots = 0;
  int scratch_stride = 0;
  std::vector<scqr3_batch_item> src;
  std::vector<BTile> tiles;
  std::vector<int> order;  // items sorted by class
  std::vector<int64_t> mat_off;  // per item: offset (doubles) of gram / rstack / racc block
  void* ws = nullptr;            // workspace the tables were uploaded to
};

namespace {
int bpad(int n) { return n <= 16 ? 16 : n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : 0; }
size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

extern "C" int scqr3_batch_plan_create(const scqr3_batch_item* items, int count, const scqr3_opts* opts,
                                       const scqr3_batch_tuning* tuning, scqr3_batch_plan** out,
                                       size_t* workspace_bytes) {
  if (!items) return -1;
  if (count < 1) return -2;
  if (opts && opts->max_passes != 0 && (opts->max_passes < 3 || opts->max_passes > SCQR3_MAX_PASSES))
    return -3;
  if (opts && opts->precision != SCQR3_PREC_FP64) return -3;
  if (opts && opts->algorithm != 0 && opts->algorithm != SCQR3_ALG_SCQR3 && opts->algorithm != SCQR3_ALG_ADAPTIVE)
    return -3;
  if (!out || !workspace_bytes) return -5;
  for (int i = 0; i < count; ++i) {
    const scqr3_batch_item& a = items[i];
    if (!a.X || !a.Q || !a.R || a.n < 1 || a.m < a.n || a.ldx < a.n || a.ldq < a.n || !a.info) return -1;
    if (!bpad(a.n)) return SCQR3_E_UNSUPPORTED;
    if ((const void*)a.Q != (const void*)a.X) {
      const char* px = (const char*)a.X;
      const char* pq = (const char*)a.Q;
      const size_t bx = sizeof(double) * (size_t)((a.m - 1) * a.ldx + a.n);
      const size_t bq = sizeof(double) * (size_t)((a.m - 1) * a.ldq + a.n);
      if (px < pq + bq && pq < px + bx) return -1;
    } else if (a.ldq != a.ldx) {
      return -1;
    }
  }
  scqr3_batch_plan* p = new (std::nothrow) scqr3_batch_plan();
  if (!p) return SCQR3_E_CUDA;
  p->count = count;
  p->max_passes = (opts && opts->max_passes) ? opts->max_passes : 6;
  if (opts) {
    p->opts = *opts;
    p->has_opts = true;
  }
  p->src.assign(items, items + count);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete p;
    return SCQR3_E_CUDA;
  }
  const int cps = (tuning && tuning->ctas_per_sm > 0) ? tuning->ctas_per_sm : 1;
  p->grid = sms * cps;
  // order: larger padded size first (longest tiles first), then by index
  p->order.resize(count);
  for (int i = 0; i < count; ++i) p->order[i] = i;
  std::stable_sort(p->order.begin(), p->order.end(),
                   [&](int a, int b) { return bpad(items[a].n) > bpad(items[b].n); });
  // tiles and per-item small matrices
  int64_t slot_off = 0, mat_off = 0;
  p->mat_off.assign(count, 0);
  for (int oi = 0; oi < count; ++oi) {
    const int i = p->order[oi];
    const int np = bpad(items[i].n);
    p->np_max = std::max(p->np_max, np);
    const int E = pk_size(np);
    const int slotc = np == 16 ? 0 : np == 32 ? 1 : np == 64 ? 2 : 3;
    int tp = (tuning && tuning->tile_panels[slotc] > 0) ? tuning->tile_panels[slotc] : 0;
    const int64_t npan = (items[i].m + batched_rows_per_panel(np) - 1) / batched_rows_per_panel(np);
    if (tp <= 0) tp = 8;  // default tile: 8 panels
    p->mat_off[i] = mat_off;
    mat_off += (E + 1) + (int64_t)E * SCQR3_MAX_PASSES + E;
    for (int64_t pb = 0; pb < npan; pb += tp) {
      BTile t;
      t.item = i;
      t.np = np;
      t.p_begin = pb;
      t.p_end = std::min<int64_t>(npan, pb + tp);
      t.slot = slot_off;
      slot_off += E + 1;
      p->tiles.push_back(t);
    }
  }
  p->ntiles = (int)p->tiles.size();
  const int Emax = pk_size(p->np_max);
  p->scratch_stride = batched_groups(p->np_max) * (Emax + 1);
  for (int s : {16, 32, 64, 128})
    if (s <= p->np_max) p->scratch_stride = std::max(p->scratch_stride, batched_groups(s) * (pk_size(s) + 1));
  size_t off = 0;
  p->off_items = off;    off = a256(off + sizeof(BItem) * count);
  p->off_tiles = off;    off = a256(off + sizeof(BTile) * p->ntiles);
  p->off_counters = off; off = a256(off + sizeof(int) * (2 * SCQR3_MAX_PASSES + 2));
  p->off_states = off;   off = a256(off + sizeof(DevState) * count);
  p->off_mats = off;     off = a256(off + sizeof(double) * (size_t)mat_off);
  p->off_scratch = off;  off = a256(off + sizeof(double) * (size_t)p->scratch_stride * p->grid);
  p->off_slots = off;    off = a256(off + sizeof(double) * (size_t)slot_off);
  p->bytes = off;
  *workspace_bytes = off;
  *out = p;
  return SCQR3_OK;
}

extern "C" int scqr3_batch_plan_upload(scqr3_batch_plan* p, void* workspace, size_t workspace_bytes,
                                       void* stream) {
  if (!p) return -1;
  if (!workspace || ((uintptr_t)workspace & 255) != 0 || workspace_bytes < p->bytes) return SCQR3_E_WORKSPACE;
  // let the kernels use their shared memory (set-up happens here, before any capture)
  if (cudaFuncSetAttribute(batched_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)batched_pass_smem()) != cudaSuccess)
    return SCQR3_E_CUDA;
  if (cudaFuncSetAttribute(batched_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)batched_chol_smem()) != cudaSuccess)
    return SCQR3_E_CUDA;
  char* ws = (char*)workspace;
  std::vector<BItem> it(p->count);
  for (int i = 0; i < p->count; ++i) {
    const scqr3_batch_item& a = p->src[i];
    BItem& b = it[i];
    const int np = bpad(a.n);
    const int E = pk_size(np);
    b.X = a.X;
    b.Q = a.Q;
    b.R = a.R;
    b.Rpass = a.Rpass;
    b.info = a.info;
    b.st = (DevState*)(ws + p->off_states) + i;
    double* mats = (double*)(ws + p->off_mats) + p->mat_off[i];
    b.gram = mats;
    b.rstack = mats + (E + 1);
    b.racc = b.rstack + (int64_t)E * SCQR3_MAX_PASSES;
    b.P.m = a.m;
    b.P.n = a.n;
    b.P.np = np;
    b.P.max_passes = p->max_passes;
    b.P.bs = 0;
    b.P.norm_x2 = 0.0;
    b.P.normb_in = 0.0;
    set_options(&b.P, p->has_opts ? &p->opts : nullptr);  // per matrix: Alg. 2's tol depends on m, n
    b.ldx = a.ldx;
    b.ldq = a.ldq;
    b.tile_lo = b.tile_hi = -1;
  }
  for (int t = 0; t < p->ntiles; ++t) {
    BItem& b = it[p->tiles[t].item];
    if (b.tile_lo < 0) b.tile_lo = t;
    b.tile_hi = t + 1;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(ws + p->off_items, it.data(), sizeof(BItem) * p->count, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return SCQR3_E_CUDA;
  if (cudaMemcpyAsync(ws + p->off_tiles, p->tiles.data(), sizeof(BTile) * p->ntiles, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return SCQR3_E_CUDA;
  // the host vectors above are freed on return: wait for the copies
  if (cudaStreamSynchronize(s) != cudaSuccess) return SCQR3_E_CUDA;
  p->ws = workspace;
  return SCQR3_OK;
}

extern "C" int scqr3_factor_batched(const scqr3_batch_plan* p, void* stream) {
  if (!p || !p->ws) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)p->ws;
  const BItem* items = (const BItem*)(ws + p->off_items);
  const BTile* tiles = (const BTile*)(ws + p->off_tiles);
  int* counters = (int*)(ws + p->off_counters);
  double* scratch = (double*)(ws + p->off_scratch);
  double* slots = (double*)(ws + p->off_slots);
  if (cudaMemsetAsync(counters, 0, sizeof(int) * (2 * SCQR3_MAX_PASSES + 2), s) != cudaSuccess) return SCQR3_E_CUDA;
  if (cudaMemsetAsync(ws + p->off_states, 0, sizeof(DevState) * p->count, s) != cudaSuccess) return SCQR3_E_CUDA;
  const size_t smem = batched_pass_smem();
  const size_t chol_smem = batched_chol_smem();
  batched_pass_kernel<<<p->grid, kThreads, smem, s>>>(items, tiles, p->ntiles, -1, counters, scratch,
                                                      p->scratch_stride, slots);
  batched_reduce_kernel<<<p->count, 256, 0, s>>>(items, tiles, slots, -1);
  batched_chol_kernel<<<p->count, 512, chol_smem, s>>>(items, 0);
  for (int k = 0; k < p->max_passes; ++k) {
    batched_pass_kernel<<<p->grid, kThreads, smem, s>>>(items, tiles, p->ntiles, k, counters + 1 + k,
                                                        scratch, p->scratch_stride, slots);
    if (k + 1 < p->max_passes) {
      batched_reduce_kernel<<<p->count, 256, 0, s>>>(items, tiles, slots, k);
      batched_chol_kernel<<<p->count, 512, chol_smem, s>>>(items, k + 1);
    }
  }
  if (cudaGetLastError() != cudaSuccess) return SCQR3_E_CUDA;
  return SCQR3_OK;
}

extern "C" void scqr3_batch_plan_destroy(scqr3_batch_plan* p) { delete p; }
