// fam_api.cu -- host side of the FAM C ABI (include/fam.h).
//
// A handle owns three padded state buffers (A: state, B and C: stage
// buffers), a device control block (time, step size, speed reduction,
// status) and one TMA descriptor per buffer.  One step is
//   stage 1: A -> B,  stage 2: B -> C,  stage 3: C -> B,  OE: B -> A,
// with U^{n,0} = A read by stages 2 and 3 (eq. 12).  The step size lives on
// the device, so steps need no host synchronisation and are captured into
// CUDA graphs.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstddef>
#include <cstring>
#include <map>
#include <string>

#include "fam_internal.cuh"

// ---------------------------------------------------------------------------
// tensor-map encoding through the driver entry point (no link to libcuda)
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

static bool pick(fam_handle* h) {
#define FAM_PK(D, P, K) \
  if (h->d == D && h->prec == P && h->k == K) return fam_pick_d##D##_p##P##_k##K(h);
#define FAM_PKK(D, P) FAM_PK(D, P, 3) FAM_PK(D, P, 4) FAM_PK(D, P, 5) FAM_PK(D, P, 6)
  FAM_PKK(1, 64) FAM_PKK(1, 32) FAM_PKK(2, 64) FAM_PKK(2, 32)
#undef FAM_PKK
#undef FAM_PK
  return false;
}

// ghost fill of a freshly uploaded state (reads interior, writes images)
template <typename T>
__global__ void fill_ghosts_kernel(T* U, const Geo geo, int np) {
  const long long n = (long long)geo.nx * geo.ny * np;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % geo.nx);
    const long long r = q / geo.nx;
    const int j = (int)(r % geo.ny);
    const int p = (int)(r / geo.ny);
    const T v = U[cell_index(geo, p, j, i)];
    store_with_ghosts(U, geo, p, j, i, v);
  }
}

// Inflow ghosts (both layers of a side, corners included): the prescribed
// averages, zero moments (Remark in Sec. 2.3).  A side with a split holds
// them only where its nearest interior row / column lies below the split.
template <typename T>
__global__ void fill_inflow_kernel(T* U, const Geo geo, int side, int nc, const double4 st) {
  const int gx = geo.px, gy = geo.rows;
  const double sv[4] = {st.x, st.y, st.z, st.w};
  const long long n = (long long)gx * gy;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(q % gx), y = (int)(q / gx);
    bool in;
    if (side == 0) in = x < G;
    else if (side == 1) in = x >= geo.nx + G && x < geo.nx + 2 * G;
    else if (side == 2) in = gy > 1 && y < G;
    else in = gy > 1 && y >= geo.ny + G && y < geo.ny + 2 * G;
    if (!in) continue;
    if (geo.bc[side] != kBcInflow) {  // a split side: only its split part
      const int along = side < 2 ? min(max(y - G, 0), geo.ny - 1) : min(max(x - G, 0), geo.nx - 1);
      if (along >= geo.split[side]) continue;
    }
    for (int c = 0; c < nc; ++c)
      for (int m = 0; m < geo.nm; ++m) U[(long long)(c * geo.nm + m) * geo.plane + q] = m == 0 ? T(sv[c]) : T(0);
  }
}

static fam_status fill_inflow(fam_handle* h) {
  for (int side = 0; side < 4; ++side) {
    if (h->geo.bc[side] != kBcInflow && h->geo.split[side] <= 0) continue;
    const double* s = h->inflow[side];
    const double4 st = make_double4(s[0], s[1], s[2], s[3]);
    for (int b = 0; b < 3; ++b) {
      if (h->prec == 64)
        fill_inflow_kernel<double><<<148 * 4, 256, 0, h->stream>>>(bufp<double>(h, b), h->geo, side, h->nc, st);
      else
        fill_inflow_kernel<float><<<148 * 4, 256, 0, h->stream>>>(bufp<float>(h, b), h->geo, side, h->nc, st);
      FAM_CUDA(h, cudaGetLastError());
    }
  }
  return FAM_OK;
}

// Front ghosts of a y-side (both layers, every column including the x-ghost
// columns): the behind state where the ghost cell's centre (x, y) has
// x < a + b y + c t, the ahead state elsewhere; zero moments.  t is the time
// of the state in U: ctl->t + w ctl->dt, w = 0, 1, 1/2, 1 for the inputs of
// stages 1, 2, 3 and of the OE (SSP-RK3 stage times).
struct FrontArgs {
  double a, b, c, x0, yb;  // yb: the side's boundary coordinate (y0 or y1)
  double behind[4], ahead[4];
  double w;                // stage-time weight of dt
};
template <typename T>
__global__ void fill_front_kernel(T* U, const Geo geo, int side, int nc, const FrontArgs f, const FamCtl* ctl) {
  // products and sums rounded one by one (no contraction), as a plain
  // evaluation of the same expressions rounds them
  const double t = __dadd_rn(ctl->t, __dmul_rn(f.w, ctl->dt));
  const int n = geo.px * G;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int x = q % geo.px, layer = q / geo.px;  // layer 0 next to the grid
    const int y = side == 2 ? G - 1 - layer : geo.ny + G + layer;
    const double xc = __dadd_rn(f.x0, __dmul_rn(x - G + 0.5, geo.dx));
    const double off = __dmul_rn(layer + 0.5, geo.dy);
    const double yc = side == 2 ? __dsub_rn(f.yb, off) : __dadd_rn(f.yb, off);
    const bool behind = xc < __dadd_rn(__dadd_rn(f.a, __dmul_rn(f.b, yc)), __dmul_rn(f.c, t));
    const long long o = (long long)y * geo.px + x;
    for (int c = 0; c < nc; ++c)
      for (int m = 0; m < geo.nm; ++m)
        U[(long long)(c * geo.nm + m) * geo.plane + o] = m == 0 ? T(behind ? f.behind[c] : f.ahead[c]) : T(0);
  }
}

static bool has_front(const fam_handle* h) {
  return h->d == 2 && (h->geo.bc[2] == kBcFront || h->geo.bc[3] == kBcFront);
}

// Rewrite the front ghosts of buffer b for the state at ctl->t + w ctl->dt.
static fam_status fill_front(fam_handle* h, int b, double w) {
  if (!has_front(h)) return FAM_OK;
  for (int side = 2; side < 4; ++side) {
    if (h->geo.bc[side] != kBcFront) continue;
    FrontArgs f;
    f.a = h->front[side][0];
    f.b = h->front[side][1];
    f.c = h->front[side][2];
    f.x0 = h->grid.x0;
    f.yb = side == 2 ? h->grid.y0 : h->grid.y1;
    for (int c = 0; c < 4; ++c) {
      f.behind[c] = h->inflow[side][c];
      f.ahead[c] = h->front_ahead[side][c];
    }
    f.w = w;
    const int blocks = (h->geo.px * G + 255) / 256;
    if (h->prec == 64)
      fill_front_kernel<double><<<blocks, 256, 0, h->stream>>>(bufp<double>(h, b), h->geo, side, h->nc, f, h->ctl);
    else
      fill_front_kernel<float><<<blocks, 256, 0, h->stream>>>(bufp<float>(h, b), h->geo, side, h->nc, f, h->ctl);
    FAM_CUDA(h, cudaGetLastError());
  }
  return FAM_OK;
}

static fam_status fill_ghosts(fam_handle* h, int b) {
  long long n = (long long)h->geo.nx * h->geo.ny * h->np;
  int blocks = (int)std::min<long long>((n + 255) / 256, 148LL * 16);
  if (h->prec == 64)
    fill_ghosts_kernel<double><<<blocks, 256, 0, h->stream>>>(bufp<double>(h, b), h->geo, h->np);
  else
    fill_ghosts_kernel<float><<<blocks, 256, 0, h->stream>>>(bufp<float>(h, b), h->geo, h->np);
  FAM_CUDA(h, cudaGetLastError());
  return FAM_OK;
}

static fam_status encode_maps(fam_handle* h) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return fail(h, FAM_E_CUDA, "cuTensorMapEncodeTiled unavailable");
  CUtensorMapDataType dt = h->prec == 64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  for (int b = 0; b < 3; ++b) {
    CUresult r;
    if (h->d == 2) {
      cuuint64_t dims[3] = {(cuuint64_t)h->geo.px, (cuuint64_t)h->geo.rows, (cuuint64_t)h->np};
      cuuint64_t strides[2] = {(cuuint64_t)h->geo.px * h->elem, (cuuint64_t)h->geo.plane * h->elem};
      cuuint32_t box[3] = {(cuuint32_t)h->ops.tx + 4, (cuuint32_t)h->ops.ty + 4, (cuuint32_t)h->np};
      cuuint32_t es[3] = {1, 1, 1};
      r = enc(&h->tm[b], dt, 3, h->buf[b], dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r == CUDA_SUCCESS) {
        cuuint32_t box_u0[3] = {(cuuint32_t)h->ops.tx + 4, (cuuint32_t)h->ops.ty, (cuuint32_t)h->np};
        r = enc(&h->tm_u0[b], dt, 3, h->buf[b], dims, strides, box_u0, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      }
    } else {
      cuuint64_t dims[2] = {(cuuint64_t)h->geo.px, (cuuint64_t)h->np};
      cuuint64_t strides[1] = {(cuuint64_t)h->geo.plane * h->elem};
      cuuint32_t box[2] = {TX1 + 4, (cuuint32_t)h->np};
      cuuint32_t es[2] = {1, 1};
      r = enc(&h->tm[b], dt, 2, h->buf[b], dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) return fail(h, FAM_E_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(r) + ")");
  }
  return FAM_OK;
}

// shared with fam_noalloc.cu
fam_status fam_internal_encode_maps(fam_handle* h) { return encode_maps(h); }
fam_status fam_internal_fill_ghosts(fam_handle* h, int b) { return fill_ghosts(h, b); }
bool fam_internal_pick(fam_handle* h) { return pick(h); }

// ---------------------------------------------------------------------------
// control block
// ---------------------------------------------------------------------------
static fam_status ctl_read(fam_handle* h, FamCtl* out) {
  FAM_CUDA(h, cudaMemcpyAsync(out, h->ctl, sizeof(FamCtl), cudaMemcpyDeviceToHost, h->stream));
  FAM_CUDA(h, cudaStreamSynchronize(h->stream));
  return FAM_OK;
}

// (Re)compute the step size from the current state A (no time advance).
static fam_status refresh_dt(fam_handle* h, double cfl, double T, bool reset_clock) {
  FamCtl c;
  fam_status s = ctl_read(h, &c);
  if (s) return s;
  if (reset_clock) {
    c.t = 0.0;
    c.step = 0;
    c.status = 0;
  }
  c.cfl = cfl;
  c.T = T;
  c.dt_max = h->dt_max;
  c.dt = 0.0;
  c.final_step = 0;
  c.dim = h->d;
  c.dx = h->geo.dx;
  c.dy = h->geo.dy;
  const double e = h->smooth_dt ? h->k / 3.0 : 1.0;
  c.dxe = std::pow(h->geo.dx, e);
  c.dye = std::pow(h->geo.dy, e);
  c.alpha_bits[0] = c.alpha_bits[1] = 0ull;
  c.blocks_done = 0;
  c.stage_bad = 0u;
  c.retry_exp = 0u;
  FAM_CUDA(h, cudaMemcpyAsync(h->ctl, &c, sizeof(FamCtl), cudaMemcpyHostToDevice, h->stream));
  FAM_CUDA(h, h->ops.alpha(h, 0));
  FAM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->cfl_set = cfl;
  h->T_set = T;
  h->dt_valid = true;
  return FAM_OK;
}

// Type-I OE: grid statistics of the averages of buffer b before the OE kernel
static fam_status enqueue_typeI(fam_handle* h, int b) {
  if (h->oe_type != 1) return FAM_OK;
  const size_t off = offsetof(FamCtl, t1_maxabs_bits);
  FAM_CUDA(h, cudaMemsetAsync(reinterpret_cast<char*>(h->ctl) + off, 0, 2 * 4 * sizeof(unsigned long long),
                              h->stream));
  const long long n = (long long)h->geo.nx * h->geo.ny;
  if (h->prec == 64) {
    typeI_partial<double, 256><<<h->t1_blocks, 256, 0, h->stream>>>(bufp<double>(h, b), h->geo, h->nc, h->nm,
                                                                    h->t1_partial, h->ctl);
    typeI_final<<<1, 32, 0, h->stream>>>(h->t1_partial, h->t1_blocks, h->nc, n, h->ctl);
    typeI_dev<double, 256><<<h->t1_blocks, 256, 0, h->stream>>>(bufp<double>(h, b), h->geo, h->nc, h->nm, h->ctl);
  } else {
    typeI_partial<float, 256><<<h->t1_blocks, 256, 0, h->stream>>>(bufp<float>(h, b), h->geo, h->nc, h->nm,
                                                                   h->t1_partial, h->ctl);
    typeI_final<<<1, 32, 0, h->stream>>>(h->t1_partial, h->t1_blocks, h->nc, n, h->ctl);
    typeI_dev<float, 256><<<h->t1_blocks, 256, 0, h->stream>>>(bufp<float>(h, b), h->geo, h->nc, h->nm, h->ctl);
  }
  FAM_CUDA(h, cudaGetLastError());
  return FAM_OK;
}

// ---------------------------------------------------------------------------
// fused final stage + OE: task list of the persistent launch
// ---------------------------------------------------------------------------
// Stage tasks in row-major tile order; each OE task right after the last
// stage task it waits for (the tiles whose cells or ghost images its 2-cell
// halo reads, halo_tiles) plus twice the launch's resident block count, so
// that the stage tasks it needs have most likely finished when it is taken.  The
// fused path needs the Type-II (or no) OE: Type I reads grid-wide statistics
// of the final stage, which exist only once every tile has finished.
static void free_fused(fam_handle* h) {
  if (h->fz_tasks) cudaFree(h->fz_tasks);
  if (h->fz_sync) cudaFree(h->fz_sync);
  h->fz_tasks = nullptr;
  h->fz_sync = nullptr;
  h->fz_ready = false;
}

static bool has_front(const fam_handle* h);
static bool use_fused(const fam_handle* h) {
  return h->fused_oe && h->d == 2 && h->oe_type != 1 && !h->pp && !has_front(h) && h->fz_ready && h->ops.fused;
}

static fam_status build_fused(fam_handle* h) {
  if (!h->fused_oe || h->d != 2 || h->fz_ready) return FAM_OK;
  if (!h->ops.fused) return fail(h, FAM_E_UNSUPPORTED, "no fused kernel for this configuration");
  free_fused(h);
  int dev = 0, sms = 0, per_sm = 0;
  FAM_CUDA(h, cudaGetDevice(&dev));
  FAM_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  FAM_CUDA(h, h->ops.fused_occupancy(&per_sm));
  if (per_sm < 1) return fail(h, FAM_E_UNSUPPORTED, "fused kernel does not fit on an SM");
  const int TX = h->ops.tx, TY = h->ops.ty;
  const int ntx = (h->geo.nx + TX - 1) / TX, nty = (h->geo.ny + TY - 1) / TY, nt = ntx * nty;
  h->fz_grid = std::min(sms * per_sm, nt);
  std::vector<std::vector<int>> after(nt);
  const int* bc = h->geo.bc;
  for (int ty = 0; ty < nty; ++ty)
    for (int tx = 0; tx < ntx; ++tx) {
      int cx[5], cy[5];
      const int mx = halo_tiles(tx, TX, h->geo.nx, bc[0], bc[1], cx);
      const int my = halo_tiles(ty, TY, h->geo.ny, bc[2], bc[3], cy);
      int last = 0;
      for (int b = 0; b < my; ++b)
        for (int a = 0; a < mx; ++a) last = std::max(last, cy[b] * ntx + cx[a]);
      after[std::min(nt - 1, last + 2 * h->fz_grid)].push_back(ty * ntx + tx);
    }
  std::vector<int> seq;
  seq.reserve(2 * (size_t)nt);
  for (int q = 0; q < nt; ++q) {
    seq.push_back(q);
    for (int t : after[q]) seq.push_back(nt + t);
  }
  FAM_CUDA(h, cudaMalloc(&h->fz_tasks, sizeof(int) * seq.size()));
  FAM_CUDA(h, cudaMalloc(&h->fz_sync, sizeof(unsigned int) * (nt + 1)));
  FAM_CUDA(h, cudaMemcpy(h->fz_tasks, seq.data(), sizeof(int) * seq.size(), cudaMemcpyHostToDevice));
  h->fz_ntasks = (int)seq.size();
  h->fz_ntiles = nt;
  h->fz_ready = true;
  return FAM_OK;
}

static fam_status enqueue_fused(fam_handle* h) {
  FAM_CUDA(h, cudaMemsetAsync(h->fz_sync, 0, sizeof(unsigned int) * (h->fz_ntiles + 1), h->stream));
  FAM_CUDA(h, h->ops.fused(h));
  return FAM_OK;
}

// BP/PP safeguard: scaling factors of the stage input (2D) and, before the
// first stage, the step size from the limited point speeds
static fam_status pp_prep(fam_handle* h, int b, bool want_dt) {
  if (!h->pp) return FAM_OK;
  FAM_CUDA(h, h->ops.pp_prep(h, b, want_dt));
  return FAM_OK;
}

// Front ghosts follow the stage times: the inputs of stages 1, 2, 3 hold the
// states at t, t + dt, t + dt/2.  The OE's input (buffer 1) keeps the front
// rows written for stage 2's input (t + dt), which is also its own time:
// the kernels write no images into a front side.
static fam_status enqueue_step(fam_handle* h) {
  if (fam_status f = fill_front(h, 0, 0.0)) return f;
  if (fam_status p = pp_prep(h, 0, true)) return p;
  FAM_CUDA(h, h->ops.stage(h, 0, 0, 1, 1));
  if (fam_status f = fill_front(h, 1, 1.0)) return f;
  if (fam_status p = pp_prep(h, 1, false)) return p;
  FAM_CUDA(h, h->ops.stage(h, 1, 0, 2, 2));
  if (use_fused(h)) return enqueue_fused(h);
  if (fam_status f = fill_front(h, 2, 0.5)) return f;
  if (fam_status p = pp_prep(h, 2, false)) return p;
  FAM_CUDA(h, h->ops.stage(h, 2, 0, 1, 3));
  fam_status s = enqueue_typeI(h, 1);
  if (s) return s;
  FAM_CUDA(h, h->ops.oe(h, 1, 0, -1.0));
  return FAM_OK;
}

static cudaEvent_t next_event(fam_handle* h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_used++];
}

// fam_step with CUDA events around each of the four launches
static fam_status enqueue_step_profiled(fam_handle* h) {
  cudaEvent_t e[5];
  for (int q = 0; q < 5; ++q) {
    e[q] = next_event(h);
    if (!e[q]) return fail(h, FAM_E_CUDA, "cudaEventCreate failed");
  }
  FAM_CUDA(h, cudaEventRecord(e[0], h->stream));
  if (fam_status f = fill_front(h, 0, 0.0)) return f;
  if (fam_status p = pp_prep(h, 0, true)) return p;
  FAM_CUDA(h, h->ops.stage(h, 0, 0, 1, 1));
  FAM_CUDA(h, cudaEventRecord(e[1], h->stream));
  if (fam_status f = fill_front(h, 1, 1.0)) return f;
  if (fam_status p = pp_prep(h, 1, false)) return p;
  FAM_CUDA(h, h->ops.stage(h, 1, 0, 2, 2));
  FAM_CUDA(h, cudaEventRecord(e[2], h->stream));
  h->prof_fused.push_back(use_fused(h) ? 1 : 0);
  if (use_fused(h)) {  // stage 3 and OE in one launch: all of it in ms[2], none in ms[3]
    fam_status s = enqueue_fused(h);
    if (s) return s;
    FAM_CUDA(h, cudaEventRecord(e[3], h->stream));
    FAM_CUDA(h, cudaEventRecord(e[4], h->stream));
    return FAM_OK;
  }
  if (fam_status f = fill_front(h, 2, 0.5)) return f;
  if (fam_status p = pp_prep(h, 2, false)) return p;
  FAM_CUDA(h, h->ops.stage(h, 2, 0, 1, 3));
  FAM_CUDA(h, cudaEventRecord(e[3], h->stream));
  fam_status s = enqueue_typeI(h, 1);
  if (s) return s;
  FAM_CUDA(h, h->ops.oe(h, 1, 0, -1.0));
  FAM_CUDA(h, cudaEventRecord(e[4], h->stream));
  return FAM_OK;
}

// One step with a prescribed step size (adjoint recomputation).  If store is
// not null, the stage inputs U^n, U^(1), U^(2) and the pre-OE state U^(3)
// are copied into store[0..3] (padded buffers).
fam_status fam_internal_step_fixed_dt(fam_handle* h, double dt, void* const* store) {
  const size_t sb = h->buf_elems * h->elem;
  FAM_CUDA(h, cudaMemcpyAsync(&h->ctl->dt, &dt, sizeof(double), cudaMemcpyHostToDevice, h->stream));
  if (store) FAM_CUDA(h, cudaMemcpyAsync(store[0], h->buf[0], sb, cudaMemcpyDeviceToDevice, h->stream));
  if (fam_status f = fill_front(h, 0, 0.0)) return f;
  if (fam_status p = pp_prep(h, 0, false)) return p;
  FAM_CUDA(h, h->ops.stage(h, 0, 0, 1, 1));
  if (store) FAM_CUDA(h, cudaMemcpyAsync(store[1], h->buf[1], sb, cudaMemcpyDeviceToDevice, h->stream));
  if (fam_status f = fill_front(h, 1, 1.0)) return f;
  if (fam_status p = pp_prep(h, 1, false)) return p;
  FAM_CUDA(h, h->ops.stage(h, 1, 0, 2, 2));
  if (store) FAM_CUDA(h, cudaMemcpyAsync(store[2], h->buf[2], sb, cudaMemcpyDeviceToDevice, h->stream));
  if (fam_status f = fill_front(h, 2, 0.5)) return f;
  if (fam_status p = pp_prep(h, 2, false)) return p;
  FAM_CUDA(h, h->ops.stage(h, 2, 0, 1, 3));
  if (store) FAM_CUDA(h, cudaMemcpyAsync(store[3], h->buf[1], sb, cudaMemcpyDeviceToDevice, h->stream));
  fam_status st = enqueue_typeI(h, 1);
  if (st) return st;
  FAM_CUDA(h, h->ops.oe(h, 1, 0, -1.0));
  return FAM_OK;
}

fam_status refresh_dt_public(fam_handle* h, double cfl) { return refresh_dt(h, cfl, 0.0, false); }

// The four sides' conditions as a whole: periodic sides come in pairs, and
// an inflow side may not meet a reflective wall (their shared corner ghosts
// have no single rule).
static fam_status check_bc(fam_handle* h) {
  const int* nb = h->geo.bc;
  for (int dir = 0; dir < h->d; ++dir)
    if ((nb[2 * dir] == kBcPeriodic) != (nb[2 * dir + 1] == kBcPeriodic))
      return fail(h, FAM_E_INVAL, "periodic conditions come in pairs; set the opposite side too");
  for (int side = 0; side < 4; ++side)
    if (h->geo.split[side] > 0 && nb[side] == kBcPeriodic)
      return fail(h, FAM_E_INVAL, "a periodic side cannot be split");
  // an inflow side next to a reflective wall: their shared corner ghosts are
  // built only where the wall's split part (fixed state) covers the corner
  if (h->d == 2)
    for (int dir = 0; dir < 2; ++dir)
      for (int s2 = 0; s2 < 2; ++s2) {
        if (nb[2 * dir + s2] != kBcInflow) continue;
        const int n_along_other = dir == 0 ? h->geo.nx : h->geo.ny;  // cells along the other direction's sides
        for (int t2 = 0; t2 < 2; ++t2) {
          const int wall = 2 * (1 - dir) + t2;
          if (nb[wall] != kBcReflective) continue;
          const bool covered = s2 == 0 ? h->geo.split[wall] > 0 : h->geo.split[wall] >= n_along_other;
          if (!covered) return fail(h, FAM_E_UNSUPPORTED, "inflow next to a reflective wall is not built");
        }
      }
  return FAM_OK;
}

static fam_status ensure_dt(fam_handle* h, double cfl, double T) {
  if (!h->have_state) return fail(h, FAM_E_STATE, "no state: call fam_set_state first");
  {
    fam_status b = check_bc(h);
    if (b) return b;
    b = build_fused(h);  // outside any stream capture: it allocates
    if (b) return b;
  }
  if (!(cfl > 0.0)) return fail(h, FAM_E_INVAL, "cfl must be positive");
  if (!h->dt_valid || cfl != h->cfl_set || T != h->T_set) return refresh_dt(h, cfl, T, false);
  return FAM_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* fam_status_string(fam_status s) {
  switch (s) {
    case FAM_OK: return "FAM_OK";
    case FAM_E_INVAL: return "FAM_E_INVAL";
    case FAM_E_NOMEM: return "FAM_E_NOMEM";
    case FAM_E_CUDA: return "FAM_E_CUDA";
    case FAM_E_NONPHYSICAL: return "FAM_E_NONPHYSICAL";
    case FAM_E_TIMEOUT: return "FAM_E_TIMEOUT";
    case FAM_E_STATE: return "FAM_E_STATE";
    case FAM_E_UNSUPPORTED: return "FAM_E_UNSUPPORTED";
  }
  return "FAM_E_?";
}

const char* fam_last_error(fam_t h) { return h ? h->err.c_str() : "null handle"; }

void fam_destroy(fam_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  free_fused(h);
  for (int b = 0; b < 3; ++b)
    if (h->buf[b]) cudaFree(h->buf[b]);
  if (h->theta) cudaFree(h->theta);
  if (h->ctl) cudaFree(h->ctl);
  if (h->t1_partial) cudaFree(h->t1_partial);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

fam_status fam_create(fam_t* out, const fam_grid* grid, int k, int equation, int bc, double gamma, int precision,
                      void* stream) {
  if (!out || !grid) return FAM_E_INVAL;
  *out = nullptr;
  if (grid->d != 1 && grid->d != 2) return FAM_E_INVAL;
  if (k < 3 || k > 6) return FAM_E_INVAL;
  if (equation < FAM_ADVECTION || equation > FAM_BUCKLEY) return FAM_E_INVAL;
  if (equation == FAM_BUCKLEY && grid->d != 1) return FAM_E_UNSUPPORTED;  // the paper's test is 1D
  if (bc != FAM_BC_PERIODIC && bc != FAM_BC_OUTFLOW) return FAM_E_INVAL;
  if (precision != 64 && precision != 32) return FAM_E_INVAL;
  if (grid->nx < 4 || (grid->d == 2 && grid->ny < 4)) return FAM_E_INVAL;
  if (!(grid->x1 > grid->x0) || (grid->d == 2 && !(grid->y1 > grid->y0))) return FAM_E_INVAL;
  if (equation == FAM_EULER && !(gamma > 1.0)) return FAM_E_INVAL;
  fam_handle* h = new fam_handle();
  h->d = grid->d;
  h->k = k;
  h->eq = equation;
  h->bc = bc;
  h->prec = precision;
  h->grid = *grid;
  h->gamma = gamma;
  h->ax = h->ay = gamma;
  if (equation == FAM_EULER) h->ax = h->ay = 1.0;
  h->nc = equation == FAM_EULER ? grid->d + 2 : 1;
  h->nm = grid->d + 1;
  h->np = h->nc * h->nm;
  h->elem = precision == 64 ? 8 : 4;
  Geo& g = h->geo;
  g.nx = grid->nx;
  g.ny = grid->d == 2 ? grid->ny : 1;
  g.px = ((g.nx + 2 * G) + 3) / 4 * 4;
  g.rows = grid->d == 2 ? g.ny + 2 * G : 1;
  g.plane = (long long)g.px * g.rows;
  g.bcx = g.bcy = bc;
  for (int q = 0; q < 4; ++q) g.bc[q] = bc;
  g.nm = h->nm;
  g.euler = equation == FAM_EULER;
  g.dx = (grid->x1 - grid->x0) / grid->nx;
  g.dy = grid->d == 2 ? (grid->y1 - grid->y0) / grid->ny : 1.0;
  g.idx = 1.0 / g.dx;
  g.idy = 1.0 / g.dy;
  bool ok = pick(h);
  if (!ok) {
    delete h;
    return FAM_E_UNSUPPORTED;
  }
  const char* fault = std::getenv("FAM_FAULT_ALLOC");
  if (fault && fault[0] == '1') {
    delete h;
    return FAM_E_NOMEM;
  }
  cudaError_t e = h->ops.prepare();
  if (e != cudaSuccess) {
    fam_destroy(h);
    return FAM_E_CUDA;
  }
  if (stream) {
    h->stream = reinterpret_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      fam_destroy(h);
      return FAM_E_CUDA;
    }
    h->own_stream = true;
  }
  h->buf_elems = (size_t)g.plane * h->np;
  for (int b = 0; b < 3; ++b) {
    if (cudaMalloc(&h->buf[b], h->buf_elems * h->elem) != cudaSuccess) {
      fam_destroy(h);
      return FAM_E_NOMEM;
    }
    cudaMemsetAsync(h->buf[b], 0, h->buf_elems * h->elem, h->stream);
  }
  if (cudaMalloc(&h->ctl, sizeof(FamCtl)) != cudaSuccess) {
    fam_destroy(h);
    return FAM_E_NOMEM;
  }
  h->t1_blocks = (int)std::max<long long>(1, std::min<long long>(((long long)g.nx * g.ny + 255) / 256, 148LL * 4));
  if (cudaMalloc(&h->t1_partial, sizeof(double) * 4 * h->t1_blocks) != cudaSuccess) {
    fam_destroy(h);
    return FAM_E_NOMEM;
  }
  cudaMemsetAsync(h->ctl, 0, sizeof(FamCtl), h->stream);
  if (encode_maps(h) != FAM_OK) {
    fam_destroy(h);
    return FAM_E_CUDA;
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    fam_destroy(h);
    return FAM_E_CUDA;
  }
  *out = h;
  return FAM_OK;
}

// Bind the 2D kernels of tile shape kTile2D[t] and re-encode the TMA boxes.
static fam_status select_tile(fam_handle* h, int t) {
  FAM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->tile2d = t;
  free_fused(h);  // the task list depends on the tile shape
  if (!pick(h)) return fail(h, FAM_E_UNSUPPORTED, "no kernels for this configuration");
  FAM_CUDA(h, h->ops.prepare());
  fam_status s = encode_maps(h);
  if (s) return s;
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  return FAM_OK;
}

fam_status fam_tune(fam_t h, double cfl, int probe_steps, const char* cache_path, int* choice) {
  if (!h) return FAM_E_INVAL;
  if (!h->have_state) return fail(h, FAM_E_STATE, "no state: call fam_set_state first");
  if (fam_status b = check_bc(h)) return b;
  if (h->d != 2) {
    if (choice) *choice = 0;
    return FAM_OK;  // 1D kernels have a single tile shape
  }
  if (probe_steps < 1) probe_steps = 1;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, dev);
  char key[512];
  std::snprintf(key, sizeof(key), "%s|2d|eq%d|k%d|p%d|%dx%d%s", prop.name, h->eq, h->k, h->prec, h->geo.nx,
                h->geo.ny, h->pp ? "|pp" : "");
  if (cache_path && cache_path[0]) {
    FILE* f = std::fopen(cache_path, "r");
    if (f) {
      char line[600];
      while (std::fgets(line, sizeof(line), f)) {
        char* tab = std::strchr(line, '\t');
        if (!tab) continue;
        *tab = 0;
        if (std::strcmp(line, key) == 0) {
          const int t = std::atoi(tab + 1);
          std::fclose(f);
          if (t < 0 || t > 5 || (t > 2 && (h->oe_type == 1 || h->pp))) break;
          if (choice) *choice = t;
          h->fused_oe = t / 3;
          fam_status st = select_tile(h, t % 3);
          if (st == FAM_OK) st = build_fused(h);
          return st;
        }
      }
      std::fclose(f);
    }
  }
  const size_t sb = h->buf_elems * h->elem;
  void* save = nullptr;
  FAM_CUDA(h, cudaMalloc(&save, sb));
  FAM_CUDA(h, cudaMemcpyAsync(save, h->buf[0], sb, cudaMemcpyDeviceToDevice, h->stream));
  FamCtl ctl_save;
  fam_status s = ctl_read(h, &ctl_save);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int fused_was = h->fused_oe;
  int best = h->tile2d + 3 * fused_was;
  float best_ms = 1e30f;
  // candidates: every tile shape, split and (Type II / no OE, no safeguard) fused
  const int nfused = (h->oe_type == 1 || h->pp) ? 1 : 2;
  for (int cand = 0; cand < 3 * nfused && s == FAM_OK; ++cand) {
    const int t = cand % 3;
    if (select_tile(h, t) != FAM_OK) continue;
    h->fused_oe = cand / 3;
    if (build_fused(h) != FAM_OK) continue;
    cudaMemcpyAsync(h->buf[0], save, sb, cudaMemcpyDeviceToDevice, h->stream);
    if (refresh_dt(h, cfl, 0.0, true) != FAM_OK) continue;
    enqueue_step(h);  // warm-up
    cudaMemcpyAsync(h->buf[0], save, sb, cudaMemcpyDeviceToDevice, h->stream);
    if (refresh_dt(h, cfl, 0.0, true) != FAM_OK) continue;
    cudaEventRecord(e0, h->stream);
    for (int q = 0; q < probe_steps; ++q) enqueue_step(h);
    cudaEventRecord(e1, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = cand;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->fused_oe = best / 3;
  fam_status s2 = select_tile(h, best % 3);
  if (s2 == FAM_OK) s2 = build_fused(h);
  cudaMemcpyAsync(h->buf[0], save, sb, cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(h->ctl, &ctl_save, sizeof(FamCtl), cudaMemcpyHostToDevice, h->stream);
  cudaStreamSynchronize(h->stream);
  cudaFree(save);
  h->dt_valid = false;
  if (s) return s;
  if (s2) return s2;
  if (cache_path && cache_path[0]) {
    FILE* f = std::fopen(cache_path, "a");
    if (f) {
      std::fprintf(f, "%s\t%d\n", key, best);
      std::fclose(f);
    }
  }
  if (choice) *choice = best;
  return FAM_OK;
}

fam_status fam_set_option(fam_t h, const char* key, double v) {
  if (!h || !key) return FAM_E_INVAL;
  std::string k(key);
  if (k == "oe_type") {
    if (v == 0.0 || v == 1.0 || v == 2.0) h->oe_type = (int)v;
    else return fail(h, FAM_E_INVAL, "oe_type must be 0, 1 or 2");
  } else if (k == "gamma_k") {
    h->gamma_k = v;
  } else if (k == "oe_jump_q6") {
    h->oe_q6 = v != 0.0;
  } else if (k == "smooth_dt") {
    h->smooth_dt = v != 0.0;
  } else if (k == "ax") {
    h->ax = v;
  } else if (k == "ay") {
    h->ay = v;
  } else if (k == "dt_max") {
    h->dt_max = v;
  } else if (k == "tile2d") {
    if (h->d != 2) return fail(h, FAM_E_INVAL, "tile2d applies to 2D grids");
    if (v != 0.0 && v != 1.0 && v != 2.0) return fail(h, FAM_E_INVAL, "tile2d must be 0, 1 or 2");
    return select_tile(h, (int)v);
  } else if (k == "pp_limiter") {
    if (v != 0.0 && v != 1.0) return fail(h, FAM_E_INVAL, "pp_limiter must be 0 or 1");
    if (v != 0.0 && h->eq != FAM_EULER && h->eq != FAM_BUCKLEY)
      return fail(h, FAM_E_UNSUPPORTED, "pp_limiter is built for the Euler and Buckley-Leverett equations");
    if (v != 0.0 && h->d == 2 && !h->theta) {
      FAM_CUDA(h, cudaStreamSynchronize(h->stream));
      if (cudaMalloc(&h->theta, 2 * (size_t)h->geo.plane * h->elem) != cudaSuccess)
        return fail(h, FAM_E_NOMEM, "no memory for the scaling factors");
      // the factors of cells -1..n are written before each use; cells further
      // out only feed faces outside the grid
      FAM_CUDA(h, cudaMemsetAsync(h->theta, 0, 2 * (size_t)h->geo.plane * h->elem, h->stream));
    }
    h->pp = (int)v;
  } else if (k == "fused_oe") {
    if (h->d != 2) return fail(h, FAM_E_INVAL, "fused_oe applies to 2D grids");
    if (v != 0.0 && v != 1.0) return fail(h, FAM_E_INVAL, "fused_oe must be 0 or 1");
    h->fused_oe = (int)v;
    free_fused(h);
  } else if (k == "profile") {
    h->profile = v != 0.0;
    h->ev_used = 0;
    h->prof_fused.clear();
    h->prof_steps = 0;
    for (double& x : h->prof_ms) x = 0.0;
    return FAM_OK;
  } else {
    return fail(h, FAM_E_INVAL, "unknown option " + k);
  }
  h->dt_valid = false;
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  return FAM_OK;
}

static fam_status copy_in(fam_handle* h, const void* U, int on_device, int b) {
  if (!U) return fail(h, FAM_E_INVAL, "null state pointer");
  const Geo& g = h->geo;
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const char* src = reinterpret_cast<const char*>(U);
  char* dst = reinterpret_cast<char*>(h->buf[b]);
  const size_t row = (size_t)g.nx * h->elem;
  const size_t src_plane = row * g.ny;
  for (int p = 0; p < h->np; ++p) {
    char* d0 = dst + ((size_t)p * g.plane + (size_t)(h->d == 2 ? G : 0) * g.px + G) * h->elem;
    FAM_CUDA(h, cudaMemcpy2DAsync(d0, (size_t)g.px * h->elem, src + p * src_plane, row, row, g.ny, kind, h->stream));
  }
  return fill_ghosts(h, b);
}

static fam_status copy_out(fam_handle* h, void* U, int on_device, int b) {
  if (!U) return fail(h, FAM_E_INVAL, "null state pointer");
  const Geo& g = h->geo;
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  char* dst = reinterpret_cast<char*>(U);
  const char* src = reinterpret_cast<const char*>(h->buf[b]);
  const size_t row = (size_t)g.nx * h->elem;
  const size_t dst_plane = row * g.ny;
  for (int p = 0; p < h->np; ++p) {
    const char* s0 = src + ((size_t)p * g.plane + (size_t)(h->d == 2 ? G : 0) * g.px + G) * h->elem;
    FAM_CUDA(h, cudaMemcpy2DAsync(dst + p * dst_plane, row, s0, (size_t)g.px * h->elem, row, g.ny, kind, h->stream));
  }
  if (!on_device) FAM_CUDA(h, cudaStreamSynchronize(h->stream));
  return FAM_OK;
}

fam_status fam_set_bc(fam_t h, int side, int bc, const double* inflow_state) {
  if (!h || side < 0 || side > 3 || bc < kBcPeriodic || bc > kBcInflow) return FAM_E_INVAL;
  if (side >= 2 && h->d == 1) return fail(h, FAM_E_INVAL, "1D grids have only the x sides");
  if (bc == kBcInflow && !inflow_state) return fail(h, FAM_E_INVAL, "inflow needs a state");
  // sides are set one at a time; the combination is checked when it is used (check_bc)
  h->geo.bc[side] = bc;
  h->geo.bcx = h->geo.bc[0];
  h->geo.bcy = h->geo.bc[2];
  free_fused(h);  // the fused task order follows the sides' ghost images
  if (bc == kBcInflow)
    for (int c = 0; c < h->nc; ++c) h->inflow[side][c] = inflow_state[c];
  fam_status s = fill_inflow(h);
  if (s) return s;
  if (h->have_state) {
    s = fill_ghosts(h, 0);
    if (s) return s;
  }
  FAM_CUDA(h, cudaStreamSynchronize(h->stream));
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  h->dt_valid = false;
  return FAM_OK;
}

// Shared tail of the side-condition setters: fixed ghosts, images, graphs.
static fam_status side_changed(fam_handle* h) {
  h->geo.bcx = h->geo.bc[0];
  h->geo.bcy = h->geo.bc[2];
  free_fused(h);
  fam_status s = fill_inflow(h);
  if (s) return s;
  if (h->have_state) {
    s = fill_ghosts(h, 0);
    if (s) return s;
  }
  FAM_CUDA(h, cudaStreamSynchronize(h->stream));
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  h->dt_valid = false;
  return FAM_OK;
}

fam_status fam_set_bc_split(fam_t h, int side, double position, const double* state) {
  if (!h || side < 0 || side > 3) return FAM_E_INVAL;
  if (side >= 2 && h->d == 1) return fail(h, FAM_E_INVAL, "1D grids have only the x sides");
  if (h->d == 1) return fail(h, FAM_E_UNSUPPORTED, "a split needs a side with more than one cell");
  if (h->geo.bc[side] == kBcPeriodic) return fail(h, FAM_E_INVAL, "a periodic side cannot be split");
  if (!state) return fail(h, FAM_E_INVAL, "a split needs a state");
  // cells along the side whose centre lies below position (the same rounding
  // as a plain evaluation of x0 + (i + 1/2) dx)
  const bool xs = side < 2;  // the x-sides run along y
  const int n = xs ? h->geo.ny : h->geo.nx;
  const double lo = xs ? h->grid.y0 : h->grid.x0;
  const double d = xs ? h->geo.dy : h->geo.dx;
  int idx = 0;
  while (idx < n && lo + (idx + 0.5) * d < position) ++idx;
  h->geo.split[side] = idx;
  for (int c = 0; c < h->nc; ++c) h->inflow[side][c] = state[c];
  return side_changed(h);
}

fam_status fam_set_bc_front(fam_t h, int side, double a, double b, double c, const double* behind,
                            const double* ahead) {
  if (!h || side < 0 || side > 3) return FAM_E_INVAL;
  if (h->d != 2 || side < 2) return fail(h, FAM_E_INVAL, "a front condition is built for the y-sides of a 2D grid");
  if (!behind || !ahead) return fail(h, FAM_E_INVAL, "a front needs both states");
  h->geo.bc[side] = kBcFront;
  h->front[side][0] = a;
  h->front[side][1] = b;
  h->front[side][2] = c;
  for (int q = 0; q < h->nc; ++q) {
    h->inflow[side][q] = behind[q];
    h->front_ahead[side][q] = ahead[q];
  }
  return side_changed(h);
}

fam_status fam_set_state(fam_t h, const void* U, int on_device) {
  if (!h) return FAM_E_INVAL;
  fam_status s = copy_in(h, U, on_device, 0);
  if (s) return s;
  h->have_state = true;
  h->dt_valid = false;
  // reset the clock; the step size is computed at the first step
  FamCtl c;
  std::memset(&c, 0, sizeof(c));
  FAM_CUDA(h, cudaMemcpyAsync(h->ctl, &c, sizeof(FamCtl), cudaMemcpyHostToDevice, h->stream));
  if (!on_device) FAM_CUDA(h, cudaStreamSynchronize(h->stream));
  return FAM_OK;
}

fam_status fam_get_state(fam_t h, void* U, int on_device) {
  if (!h) return FAM_E_INVAL;
  if (!h->have_state) return fail(h, FAM_E_STATE, "no state");
  return copy_out(h, U, on_device, 0);
}

fam_status fam_step(fam_t h, double cfl) {
  if (!h) return FAM_E_INVAL;
  fam_status s = ensure_dt(h, cfl, h->T_set);
  if (s) return s;
  return h->profile ? enqueue_step_profiled(h) : enqueue_step(h);
}

fam_status fam_run_steps(fam_t h, long nsteps, double cfl) {
  if (!h) return FAM_E_INVAL;
  if (nsteps < 0) return fail(h, FAM_E_INVAL, "nsteps < 0");
  fam_status s = ensure_dt(h, cfl, h->T_set);
  if (s) return s;
  if (nsteps == 0) return FAM_OK;
  auto it = h->graphs.find(nsteps);
  if (it == h->graphs.end()) {
    cudaGraph_t graph;
    FAM_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    fam_status es = FAM_OK;
    for (long q = 0; q < nsteps && es == FAM_OK; ++q) es = enqueue_step(h);
    cudaError_t ce = cudaStreamEndCapture(h->stream, &graph);
    if (es) return es;
    if (ce != cudaSuccess) return cuda_fail(h, ce, "cudaStreamEndCapture");
    cudaGraphExec_t exec;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return cuda_fail(h, ce, "cudaGraphInstantiate");
    it = h->graphs.emplace(nsteps, exec).first;
  }
  FAM_CUDA(h, cudaGraphLaunch(it->second, h->stream));
  return FAM_OK;
}

fam_status fam_run_fixed(fam_t h, long nsteps, const double* dts) {
  if (!h || (nsteps > 0 && !dts)) return FAM_E_INVAL;
  if (!h->have_state) return fail(h, FAM_E_STATE, "no state: call fam_set_state first");
  if (fam_status b = check_bc(h)) return b;
  for (long q = 0; q < nsteps; ++q) {
    if (!(dts[q] > 0.0)) return fail(h, FAM_E_INVAL, "step sizes must be positive");
    fam_status s = fam_internal_step_fixed_dt(h, dts[q], nullptr);
    if (s) return s;
  }
  h->dt_valid = false;  // the next CFL step recomputes its size from the state
  return FAM_OK;
}

fam_status fam_sync(fam_t h) {
  if (!h) return FAM_E_INVAL;
  FamCtl c;
  fam_status s = ctl_read(h, &c);
  if (s) return s;
  if (c.status & kStatusTimeout) {
    static const char* kinds[] = {"?", "tile copy", "U^n copy", "tile flag"};
    char msg[200];
    std::snprintf(msg, sizeof(msg), "a kernel's bounded wait timed out (%s; task %u, waited for %u, phase %u)",
                  kinds[c.wait_where <= 3u ? c.wait_where : 0u], c.wait_task, c.wait_dep, c.wait_phase);
    return fail(h, FAM_E_TIMEOUT, msg);
  }
  if (c.status & (kStatusNonFinite | kStatusNonPhysical))
    return fail(h, FAM_E_NONPHYSICAL, (c.status & kStatusNonFinite) ? "non-finite state" : "non-physical state");
  return FAM_OK;
}

fam_status fam_run(fam_t h, double T, double cfl, long max_steps, long* nsteps_out) {
  if (!h) return FAM_E_INVAL;
  if (!(T > 0.0)) return fail(h, FAM_E_INVAL, "T must be positive");
  fam_status s = ensure_dt(h, cfl, T);
  if (s) return s;
  FamCtl c;
  s = ctl_read(h, &c);
  if (s) return s;
  const unsigned long long start = c.step;
  long done = 0;
  const long chunk = 16;
  while (c.dt > 0.0 && (max_steps <= 0 || done < max_steps)) {
    long n = chunk;
    if (max_steps > 0 && max_steps - done < n) n = max_steps - done;
    s = fam_run_steps(h, n, cfl);
    if (s) return s;
    s = fam_sync(h);
    if (s) return s;
    s = ctl_read(h, &c);
    if (s) return s;
    done = (long)(c.step - start);
  }
  if (nsteps_out) *nsteps_out = (long)(c.step - start);
  return FAM_OK;
}

fam_status fam_time(fam_t h, double* t, double* dt_next, long* steps) {
  if (!h) return FAM_E_INVAL;
  FamCtl c;
  fam_status s = ctl_read(h, &c);
  if (s) return s;
  if (t) *t = c.t;
  if (dt_next) *dt_next = c.dt;
  if (steps) *steps = (long)c.step;
  return FAM_OK;
}

fam_status fam_rejected_steps(fam_t h, unsigned long long* count) {
  if (!h || !count) return FAM_E_INVAL;
  FamCtl c;
  fam_status s = ctl_read(h, &c);
  if (s) return s;
  *count = c.rejected;
  return FAM_OK;
}

fam_status fam_nonphysical_traces(fam_t h, unsigned long long* count) {
  if (!h || !count) return FAM_E_INVAL;
  FamCtl c;
  fam_status s = ctl_read(h, &c);
  if (s) return s;
  *count = c.ntrace;
  return FAM_OK;
}

fam_status fam_profile(fam_t h, double* ms, long* nsteps) {
  if (!h || !ms) return FAM_E_INVAL;
  FAM_CUDA(h, cudaStreamSynchronize(h->stream));
  for (size_t b = 0; b + 5 <= h->ev_used; b += 5) {
    const bool fused = b / 5 < h->prof_fused.size() && h->prof_fused[b / 5];
    for (int q = 0; q < (fused ? 3 : 4); ++q) {
      float t = 0.f;
      FAM_CUDA(h, cudaEventElapsedTime(&t, h->ev_pool[b + q], h->ev_pool[b + q + 1]));
      h->prof_ms[q] += t;
    }
    h->prof_steps += 1;
  }
  h->ev_used = 0;
  h->prof_fused.clear();
  for (int q = 0; q < 4; ++q) ms[q] = h->prof_ms[q];
  if (nsteps) *nsteps = h->prof_steps;
  return FAM_OK;
}

fam_status fam_residual(fam_t h, const void* U, void* R, int on_device) {
  if (!h) return FAM_E_INVAL;
  if (fam_status b = check_bc(h)) return b;
  fam_status s = copy_in(h, U, on_device, 1);
  if (s) return s;
  if ((s = fill_front(h, 1, 0.0))) return s;  // the state at the handle's current time
  if ((s = pp_prep(h, 1, false))) return s;
  FAM_CUDA(h, h->ops.stage(h, 1, 1, 2, 0));
  return copy_out(h, R, on_device, 2);
}

fam_status fam_oe(fam_t h, double dt, const void* U, void* Uout, int on_device) {
  if (!h) return FAM_E_INVAL;
  if (!(dt >= 0.0)) return fail(h, FAM_E_INVAL, "dt must be >= 0");
  dt = dt + 0.0;  // -0 -> +0: the kernels tell an override (>= 0) by the sign bit
  if (fam_status b = check_bc(h)) return b;
  fam_status s = copy_in(h, U, on_device, 1);
  if (s) return s;
  if ((s = fill_front(h, 1, 0.0))) return s;  // the state at the handle's current time
  s = enqueue_typeI(h, 1);
  if (s) return s;
  FAM_CUDA(h, h->ops.oe(h, 1, 2, dt));
  s = copy_out(h, Uout, on_device, 2);
  if (s) return s;
  FAM_CUDA(h, cudaStreamSynchronize(h->stream));
  return FAM_OK;
}

}  // extern "C"
