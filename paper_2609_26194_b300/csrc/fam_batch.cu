// fam_batch.cu -- many independent FAM problems in one persistent launch.
//
// Instances of uneven size and order k_i (3..6) share three packed state
// buffers (A state, B and C stage buffers; instance i at element offset
// off_i, SoA planes of padded pitch px_i).  1D: their cells are cut into tiles
// of TX cells; one cooperative persistent kernel (below) walks the tile list
// for each pass of a time step -- stage 1, 2, 3 (eq. 3 / 12) and OE (eq. 9 /
// 1dOE_system) -- with a bounded grid barrier between passes, and a per-
// instance step-size pass (Sec. 4 CFL rule with the instance's own maximum
// Rusanov speed) at the end of each step.  The arithmetic per tile is the
// same device code as the single-problem kernels (stage1d_tile,
// oe1d_tile), so every instance evolves bit for bit as it would alone.
// 2D (Euler): the same scheme over TX x TY tiles, kernel in fam_batch2d.cu.
//
// Tile shape and blocks per SM are chosen by fam_batch_tune(), which times
// each candidate on the handle's own data and can cache the choice in a file.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/fam.h"
#include "fam_batch.cuh"
#include "fam_kernels1d.cuh"

using namespace fam;

namespace {

template <typename T, int TX>
__device__ __forceinline__ void load_tile_plain(T* tile, const T* __restrict__ in, const BatchInst& I, int np,
                                                int x0) {
  constexpr int HX = TX + 4;
  for (int q = threadIdx.x; q < np * HX; q += TX) {
    const int p = q / HX, c = q - p * HX, col = x0 + c;
    tile[q] = col < I.px ? in[I.off + (long long)p * I.px + col] : T(0);
  }
}

__device__ __forceinline__ Geo geo_of(const BatchInst& I, int bc) {
  Geo g;
  g.nx = I.nx;
  g.ny = 1;
  g.px = I.px;
  g.rows = 1;
  g.plane = I.px;
  g.bcx = g.bcy = bc;
  for (int q = 0; q < 4; ++q) g.bc[q] = bc;
  g.nm = 2;
  g.euler = 1;
  g.dx = I.dx;
  g.dy = 1.0;
  g.idx = I.idx;
  g.idy = 1.0;
  return g;
}

// BP/PP safeguard (Euler): the largest spectral radius at the check points
// of the limited reconstructions of the cells of every tile of A, into each
// instance's speed maximum (the safeguard's CFL speeds; fam_pp.cuh).
template <typename T, class PH, int TX, int NP, int HX>
__device__ __forceinline__ void pp_speed_pass(const BatchInst* __restrict__ inst, const int4* __restrict__ tiles,
                                              int ntiles, const T* A, BatchCtl* ictl, const PH& ph, T* tile,
                                              double* red) {
  constexpr int NC = PH::NC;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int4 td = tiles[t];
    const BatchInst I = inst[td.x];
    __syncthreads();
    load_tile_plain<T, TX>(tile, A, I, NP, td.y);
    __syncthreads();
    T m = T(0);
    if (td.y + (int)threadIdx.x < I.nx) {
      const int hx = threadIdx.x + 2;
      auto cell = [&](auto kc) {
        constexpr int K = decltype(kc)::value;
        T cf[NC][K];
#pragma unroll
        for (int c = 0; c < NC; ++c) coef1d<T, K, HX>(tile, c, hx, cf[c]);
        T avg[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) avg[c] = cf[c][0];
        T tr, tt;
        pp_limit_1d<T, K, NC>(cf, ph.gm1, tr, tt);
        m = ph.speed_x(avg);
        pp_points_1d<T, K, NC>(cf, [&](const T* u) { m = max_nonneg(m, ph.speed_x(u)); });
      };
      switch (I.k) {
        case 3: cell(std::integral_constant<int, 3>{}); break;
        case 4: cell(std::integral_constant<int, 4>{}); break;
        case 5: cell(std::integral_constant<int, 5>{}); break;
        default: cell(std::integral_constant<int, 6>{}); break;
      }
    }
    const T bm = block_max<TX>(m, red);
    if (threadIdx.x == 0) atomic_max_nonneg(&ictl[td.x].alpha_bits, (double)bm);
  }
}

// PP: the BP/PP safeguard (Euler) scales every stage's reconstructions and
// sets the step sizes from the limited point speeds.
template <typename T, class PH, int TX, bool PP = false>
__global__ void __launch_bounds__(TX) batched1d_run(const BatchInst* __restrict__ inst,
                                                    const int4* __restrict__ tiles, int ntiles, int ninst,
                                                    T* A, T* B, T* C, BatchCtl* ictl, BatchGlobal* g, const PH ph,
                                                    int nsteps, double cfl, int oe_type, int bc, int init) {
  constexpr int NC = PH::NC, NP = 2 * NC, HX = TX + 4;
  __shared__ __align__(16) T tile[NP * HX];
  __shared__ __align__(16) T faces[2 * (TX + 2) * NC + (TX + 2)];
  __shared__ double red[64];
  const unsigned int nb = gridDim.x;

  if (init) {
    // speeds at the cell averages of A -> first step size of every instance
    for (int t = blockIdx.x; t < ntiles; t += nb) {
      const int4 td = tiles[t];
      const BatchInst I = inst[td.x];
      double m = 0.0;
      const int i = td.y + threadIdx.x;
      if (i < I.nx) {
        T u[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) u[c] = A[I.off + (long long)(c * 2) * I.px + G + i];
        m = (double)ph.speed_x(u);
      }
      m = block_max<TX>(m, red);
      if (threadIdx.x == 0) atomic_max_nonneg(&ictl[td.x].alpha_bits, m);
    }
    if constexpr (PP && NC == 3) pp_speed_pass<T, PH, TX, NP, HX>(inst, tiles, ntiles, A, ictl, ph, tile, red);
    if (!grid_barrier(g, nb)) return;
    for (int i = blockIdx.x * TX + threadIdx.x; i < ninst; i += nb * TX) {
      const double a = __longlong_as_double((long long)ictl[i].alpha_bits);
      double dt = cfl * inst[i].dx / a;
      if (!(dt > 0.0) || !isfinite(dt)) {
        dt = 0.0;
        ictl[i].status |= kStatusNonFinite;
        atomicOr(&g->status, kStatusNonFinite);
      }
      ictl[i].dt = dt;
      ictl[i].alpha_bits = 0ull;
    }
    if (!grid_barrier(g, nb)) return;
  }

  for (int s = 0; s < nsteps; ++s) {
    for (int pass = 1; pass <= 4; ++pass) {
      const T* in = pass == 1 ? A : pass == 2 ? B : pass == 3 ? C : B;
      T* out = pass == 1 ? B : pass == 2 ? C : pass == 3 ? B : A;
      for (int t = blockIdx.x; t < ntiles; t += nb) {
        const int4 td = tiles[t];
        const BatchInst I = inst[td.x];
        const double dtd = ictl[td.x].dt;
        if (!(dtd > 0.0)) continue;
        if constexpr (PP) {
          // a stage that left the admissible set discards the instance's
          // step: its later stages and its OE skip it (A keeps U^n).  Only
          // the bits of earlier passes are read, which the grid barrier has
          // settled, so every thread of the block takes the same branch.
          const unsigned int bad = *reinterpret_cast<volatile const unsigned int*>(&ictl[td.x].stage_bad);
          if ((bad & ((1u << pass) - 1u)) != 0u) continue;
        }
        __syncthreads();
        load_tile_plain<T, TX>(tile, in, I, NP, td.y);
        __syncthreads();
        const Geo geo = geo_of(I, bc);
        const T dt = T(dtd);
        if (pass < 4) {
          T* fL = faces;
          T* fR = faces + (TX + 1) * NC;
          const T* U0 = A + I.off;
          T* Uo = out + I.off;
          unsigned long long* nt = &ictl[td.x].ntrace;
          unsigned int* sb = PP ? &ictl[td.x].stage_bad : nullptr;
          switch (I.k) {
            case 3: stage1d_tile<T, 3, PH, TX, PP>(tile, fL, fR, U0, Uo, geo, ph, dt, pass, td.y, nt, sb); break;
            case 4: stage1d_tile<T, 4, PH, TX, PP>(tile, fL, fR, U0, Uo, geo, ph, dt, pass, td.y, nt, sb); break;
            case 5: stage1d_tile<T, 5, PH, TX, PP>(tile, fL, fR, U0, Uo, geo, ph, dt, pass, td.y, nt, sb); break;
            default: stage1d_tile<T, 6, PH, TX, PP>(tile, fL, fR, U0, Uo, geo, ph, dt, pass, td.y, nt, sb); break;
          }
        } else {
          T* tr = faces;
          T* sp = faces + 2 * (TX + 2) * NC;
          T* Uo = out + I.off;
          const T gk = T(I.gamma_k);
          T m;
          switch (I.k) {
            case 3: m = oe1d_tile<T, 3, PH, TX>(tile, tr, sp, Uo, geo, ph, dt, oe_type, gk, td.y, &ictl[td.x].status); break;
            case 4: m = oe1d_tile<T, 4, PH, TX>(tile, tr, sp, Uo, geo, ph, dt, oe_type, gk, td.y, &ictl[td.x].status); break;
            case 5: m = oe1d_tile<T, 5, PH, TX>(tile, tr, sp, Uo, geo, ph, dt, oe_type, gk, td.y, &ictl[td.x].status); break;
            default: m = oe1d_tile<T, 6, PH, TX>(tile, tr, sp, Uo, geo, ph, dt, oe_type, gk, td.y, &ictl[td.x].status); break;
          }
          m = block_max<TX>(m, red);
          if (threadIdx.x == 0) atomic_max_nonneg(&ictl[td.x].alpha_bits, (double)m);
        }
      }
      if (!grid_barrier(g, nb)) return;
    }
    if constexpr (PP && NC == 3) {
      pp_speed_pass<T, PH, TX, NP, HX>(inst, tiles, ntiles, A, ictl, ph, tile, red);
      if (!grid_barrier(g, nb)) return;
    }
    // per-instance clock and next step size
    for (int i = blockIdx.x * TX + threadIdx.x; i < ninst; i += nb * TX) {
      BatchCtl c = ictl[i];
      if (c.dt > 0.0) {
        if (PP && c.stage_bad != 0u) {
          // discarded step: the clock stays and the retry takes half the
          // size (U^n's speeds are those the discarded size came from)
          c.stage_bad = 0u;
          c.rejected += 1ull;
          if (++c.retry_exp > 30u) {  // the step that could not be taken stops the instance
            c.status |= kStatusNonPhysical;
            if (c.bad_step == 0ull) c.bad_step = c.steps + 1ull;
          }
          c.dt = 0.5 * c.dt;
        } else {
          c.t += c.dt;
          c.steps += 1;
          c.retry_exp = 0u;
          const double a = __longlong_as_double((long long)c.alpha_bits);
          double dt = cfl * inst[i].dx / a;
          if (!(dt > 0.0) || !isfinite(dt)) { dt = 0.0; c.status |= kStatusNonFinite; }
          c.dt = dt;
        }
        close_instance_step(c, &g->status);
      }
      c.alpha_bits = 0ull;
      ictl[i] = c;
    }
    if (!grid_barrier(g, nb)) return;
  }
}

template <typename T, int TX>
__global__ void fill_ghosts_batch(T* U, const BatchInst* inst, int ninst, int np, int bc) {
  for (int i = blockIdx.x; i < ninst; i += gridDim.x) {
    const BatchInst I = inst[i];
    Geo geo;
    geo.nx = I.nx; geo.ny = 1; geo.px = I.px; geo.rows = 1; geo.plane = I.px; geo.bcx = geo.bcy = bc;
    for (int q = 0; q < 4; ++q) geo.bc[q] = bc;
    geo.nm = 2;
    geo.euler = 1;
    geo.dx = I.dx; geo.dy = 1.0; geo.idx = I.idx; geo.idy = 1.0;
    for (int q = threadIdx.x; q < np * I.nx; q += blockDim.x) {
      const int p = q / I.nx, c = q % I.nx;
      const T v = U[I.off + (long long)p * I.px + G + c];
      store_with_ghosts(U + I.off, geo, p, 0, c, v);
    }
  }
}

template <typename T>
__global__ void fill_ghosts_batch2d(T* U, const BatchInst* inst, int ninst, int np, int bc) {
  for (int i = blockIdx.x; i < ninst; i += gridDim.x) {
    const BatchInst I = inst[i];
    Geo geo;
    geo.nx = I.nx; geo.ny = I.ny; geo.px = I.px; geo.rows = I.rows; geo.plane = I.plane; geo.bcx = geo.bcy = bc;
    for (int q = 0; q < 4; ++q) geo.bc[q] = bc;
    geo.nm = 3;
    geo.euler = 1;
    geo.dx = I.dx; geo.dy = I.dy; geo.idx = I.idx; geo.idy = I.idy;
    const long long n = (long long)np * I.nx * I.ny;
    for (long long q = threadIdx.x; q < n; q += blockDim.x) {
      const int c = (int)(q % I.nx);
      const long long r = q / I.nx;
      const int j = (int)(r % I.ny), p = (int)(r / I.ny);
      const T v = U[I.off + cell_index(geo, p, j, c)];
      store_with_ghosts(U + I.off, geo, p, j, c, v);
    }
  }
}

// 2D tile shapes, the same as the single-problem 2D kernels'
constexpr int kBatchTile2D[3][2] = {{32, 8}, {32, 4}, {16, 8}};

// Set the barrier's wait limit and test hook (leaves the barrier state alone).
__global__ void batch_glob_limits(BatchGlobal* g, unsigned long long wait_ns, unsigned int extra) {
  g->wait_ns = wait_ns;
  g->extra = extra;
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct fam_batch {
  int d = 1;       // 1 or 2
  int tile2d = 2;  // 2D: index into kBatchTile2D
  int n = 0, eq = FAM_EULER, bc = FAM_BC_OUTFLOW, prec = 64, nc = 3, np = 6;
  double gamma = 1.4, ax = 1.0;
  double gamma_k = 0.0;
  int oe_type = 2;
  size_t elem = 8;
  std::vector<int> nx, ny, k;
  std::vector<BatchInst> hinst;
  long long total = 0;  // elements per buffer
  long long cells = 0;
  BatchInst* dinst = nullptr;
  Geo* dgeo = nullptr;  // 2D: per-instance geometry for the tile code
  int4* dtiles = nullptr;
  int ntiles = 0;
  int tile_x = 128;
  int blocks_per_sm = 0;  // 0: occupancy maximum
  int grid = 0;
  int pp = 0;                      // BP/PP safeguard (1D Euler)
  unsigned long long wait_ns = 0;  // grid-barrier wait limit (0: kWaitLimitNs)
  unsigned int barrier_extra = 0;  // test hook: arrivals the barrier waits for in vain
  void* buf[3] = {nullptr, nullptr, nullptr};
  BatchCtl* ictl = nullptr;
  BatchGlobal* glob = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool have_state = false, dt_valid = false;
  double cfl_set = -1.0;
  std::vector<std::pair<std::pair<long, double>, cudaGraphExec_t>> graphs;
  std::string err;
};

static fam_status bfail(fam_batch* h, fam_status s, const std::string& m) {
  if (h) h->err = m;
  return s;
}
#define FAMB_CUDA(h, call)                                                                     \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return bfail(h, FAM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T, class PH, int TX>
static cudaError_t launch_run(fam_batch* h, const PH& ph, long nsteps, double cfl, int init, bool query_only,
                              int* grid_out) {
  auto fn = batched1d_run<T, PH, TX>;
  if constexpr (PH::NC == 3)
    if (h->pp) fn = batched1d_run<T, PH, TX, true>;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, TX, 0);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorLaunchOutOfResources;
  int per_sm = h->blocks_per_sm > 0 ? std::min(h->blocks_per_sm, occ) : occ;
  int grid = std::max(1, std::min(sms * per_sm, h->ntiles));
  if (grid_out) *grid_out = grid;
  if (query_only) return cudaSuccess;
  T* A = reinterpret_cast<T*>(h->buf[0]);
  T* B = reinterpret_cast<T*>(h->buf[1]);
  T* C = reinterpret_cast<T*>(h->buf[2]);
  int ntiles = h->ntiles, ninst = h->n, ns = (int)nsteps, oe = h->oe_type, bc = h->bc;
  const BatchInst* di = h->dinst;
  const int4* dtl = h->dtiles;
  BatchCtl* ic = h->ictl;
  BatchGlobal* gl = h->glob;
  void* args[] = {(void*)&di, (void*)&dtl, (void*)&ntiles, (void*)&ninst, (void*)&A, (void*)&B, (void*)&C,
                  (void*)&ic, (void*)&gl, (void*)&ph, (void*)&ns, (void*)&cfl, (void*)&oe, (void*)&bc,
                  (void*)&init};
  return cudaLaunchCooperativeKernel((void*)fn, dim3(grid), dim3(TX), args, 0, h->stream);
}

template <typename T, class PH>
static cudaError_t launch_tx(fam_batch* h, const PH& ph, long nsteps, double cfl, int init, bool q, int* g) {
  switch (h->tile_x) {
    case 64: return launch_run<T, PH, 64>(h, ph, nsteps, cfl, init, q, g);
    case 256: return launch_run<T, PH, 256>(h, ph, nsteps, cfl, init, q, g);
    default: return launch_run<T, PH, 128>(h, ph, nsteps, cfl, init, q, g);
  }
}

static cudaError_t launch(fam_batch* h, long nsteps, double cfl, int init, bool q = false, int* g = nullptr) {
  const double gm = h->gamma;
  if (h->d == 2) {
    Batch2DArgs a{h->dinst, h->dgeo, h->dtiles, h->ntiles, h->n, h->buf[0], h->buf[1], h->buf[2], h->ictl, h->glob,
                  h->eq, gm, (int)nsteps, cfl, h->oe_type, h->bc, init};
    return h->prec == 64 ? fam_batch2d_launch_p64(a, h->tile2d, h->blocks_per_sm, q, g, h->stream)
                         : fam_batch2d_launch_p32(a, h->tile2d, h->blocks_per_sm, q, g, h->stream);
  }
  if (h->prec == 64) {
    switch (h->eq) {
      case FAM_ADVECTION: return launch_tx<double>(h, Advection1D<double>{h->ax}, nsteps, cfl, init, q, g);
      case FAM_BURGERS: return launch_tx<double>(h, Burgers1D<double>{}, nsteps, cfl, init, q, g);
      default: return launch_tx<double>(h, Euler1D<double>{gm, gm - 1.0, 0.5 * (gm - 1.0)}, nsteps, cfl, init, q, g);
    }
  }
  switch (h->eq) {
    case FAM_ADVECTION: return launch_tx<float>(h, Advection1D<float>{(float)h->ax}, nsteps, cfl, init, q, g);
    case FAM_BURGERS: return launch_tx<float>(h, Burgers1D<float>{}, nsteps, cfl, init, q, g);
    default:
      return launch_tx<float>(h, Euler1D<float>{(float)gm, (float)(gm - 1.0), (float)(0.5 * (gm - 1.0))}, nsteps,
                              cfl, init, q, g);
  }
}

static fam_status build_tiles(fam_batch* h) {
  std::vector<int4> tl;
  std::vector<int> order(h->n);
  for (int i = 0; i < h->n; ++i) order[i] = i;
  // costliest orders first so that every round of the block-cyclic walk has
  // tiles of similar cost
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return h->k[a] > h->k[b]; });
  if (h->d == 1) {
    for (int i : order)
      for (int x0 = 0; x0 < h->nx[i]; x0 += h->tile_x) tl.push_back(make_int4(i, x0, 0, 0));
  } else {
    const int tx = kBatchTile2D[h->tile2d][0], ty = kBatchTile2D[h->tile2d][1];
    for (int i : order)
      for (int y0 = 0; y0 < h->ny[i]; y0 += ty)
        for (int x0 = 0; x0 < h->nx[i]; x0 += tx) tl.push_back(make_int4(i, x0, y0, 0));
  }
  h->ntiles = (int)tl.size();
  if (h->dtiles) cudaFree(h->dtiles);
  h->dtiles = nullptr;
  FAMB_CUDA(h, cudaMalloc(&h->dtiles, sizeof(int4) * tl.size()));
  FAMB_CUDA(h, cudaMemcpy(h->dtiles, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice));
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  return FAM_OK;
}

static fam_status fill_ghosts(fam_batch* h, int b) {
  if (h->d == 2) {
    if (h->prec == 64)
      fill_ghosts_batch2d<double><<<std::min(h->n, 4096), 256, 0, h->stream>>>(
          reinterpret_cast<double*>(h->buf[b]), h->dinst, h->n, h->np, h->bc);
    else
      fill_ghosts_batch2d<float><<<std::min(h->n, 4096), 256, 0, h->stream>>>(
          reinterpret_cast<float*>(h->buf[b]), h->dinst, h->n, h->np, h->bc);
    FAMB_CUDA(h, cudaGetLastError());
    return FAM_OK;
  }
  if (h->prec == 64)
    fill_ghosts_batch<double, 256><<<std::min(h->n, 4096), 256, 0, h->stream>>>(
        reinterpret_cast<double*>(h->buf[b]), h->dinst, h->n, h->np, h->bc);
  else
    fill_ghosts_batch<float, 256><<<std::min(h->n, 4096), 256, 0, h->stream>>>(
        reinterpret_cast<float*>(h->buf[b]), h->dinst, h->n, h->np, h->bc);
  FAMB_CUDA(h, cudaGetLastError());
  return FAM_OK;
}

static fam_status reset_clock(fam_batch* h) {
  FAMB_CUDA(h, cudaMemsetAsync(h->ictl, 0, sizeof(BatchCtl) * h->n, h->stream));
  FAMB_CUDA(h, cudaMemsetAsync(h->glob, 0, sizeof(BatchGlobal), h->stream));
  batch_glob_limits<<<1, 1, 0, h->stream>>>(h->glob, h->wait_ns, h->barrier_extra);
  FAMB_CUDA(h, cudaGetLastError());
  return FAM_OK;
}

static fam_status ensure_init(fam_batch* h, double cfl) {
  if (!h->have_state) return bfail(h, FAM_E_STATE, "no state");
  if (!(cfl > 0.0)) return bfail(h, FAM_E_INVAL, "cfl must be positive");
  if (h->dt_valid && cfl == h->cfl_set) return FAM_OK;
  // step sizes from the current averages, no step
  FAMB_CUDA(h, launch(h, 0, cfl, 1));
  FAMB_CUDA(h, cudaStreamSynchronize(h->stream));
  h->dt_valid = true;
  h->cfl_set = cfl;
  return FAM_OK;
}

extern "C" {

static fam_status create_batch(fam_batch_t* out, int d, int n_inst, const int* nx, const int* ny, const int* k,
                               double x0, double x1, double y0, double y1, int equation, int bc, double gamma,
                               int precision, void* stream) {
  if (!out || !nx || !k || n_inst <= 0 || (d == 2 && !ny)) return FAM_E_INVAL;
  *out = nullptr;
  if (equation < FAM_ADVECTION || equation > FAM_EULER) return FAM_E_INVAL;
  if (d == 2 && equation != FAM_EULER) return FAM_E_UNSUPPORTED;
  if (bc != FAM_BC_PERIODIC && bc != FAM_BC_OUTFLOW) return FAM_E_INVAL;
  if (precision != 64 && precision != 32) return FAM_E_INVAL;
  if (!(x1 > x0) || (d == 2 && !(y1 > y0))) return FAM_E_INVAL;
  if (equation == FAM_EULER && !(gamma > 1.0)) return FAM_E_INVAL;
  for (int i = 0; i < n_inst; ++i)
    if (nx[i] < 4 || (d == 2 && ny[i] < 4) || k[i] < 3 || k[i] > 6) return FAM_E_INVAL;
  const char* fault = std::getenv("FAM_FAULT_ALLOC");
  if (fault && fault[0] == '1') return FAM_E_NOMEM;
  fam_batch* h = new fam_batch();
  h->d = d;
  h->n = n_inst;
  h->eq = equation;
  h->bc = bc;
  h->prec = precision;
  h->gamma = gamma;
  h->ax = equation == FAM_ADVECTION ? gamma : 1.0;
  h->nc = equation == FAM_EULER ? d + 2 : 1;
  h->np = (d + 1) * h->nc;
  h->elem = precision == 64 ? 8 : 4;
  h->nx.assign(nx, nx + n_inst);
  h->ny.assign(n_inst, 1);
  if (d == 2) h->ny.assign(ny, ny + n_inst);
  h->k.assign(k, k + n_inst);
  long long off = 0;
  for (int i = 0; i < n_inst; ++i) {
    BatchInst I{};
    I.off = off;
    I.nx = nx[i];
    I.ny = h->ny[i];
    I.px = ((nx[i] + 2 * G) + 3) / 4 * 4;
    I.rows = d == 2 ? h->ny[i] + 2 * G : 1;
    I.plane = (long long)I.px * I.rows;
    I.k = k[i];
    I.dx = (x1 - x0) / nx[i];
    I.idx = 1.0 / I.dx;
    I.dy = d == 2 ? (y1 - y0) / h->ny[i] : 1.0;
    I.idy = 1.0 / I.dy;
    // default OE coefficient gamma_k per order and dimension (Sec. 4)
    I.gamma_k = k[i] <= 4 ? 25.0 : (d == 2 ? 15.0 : 12.5);
    off += I.plane * h->np;
    h->cells += (long long)nx[i] * h->ny[i];
    h->hinst.push_back(I);
  }
  h->total = off;
  auto bail = [&](fam_status s) {
    fam_batch_destroy(h);
    return s;
  };
  if (stream) {
    h->stream = reinterpret_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(FAM_E_CUDA);
    h->own_stream = true;
  }
  for (int b = 0; b < 3; ++b) {
    if (cudaMalloc(&h->buf[b], h->total * h->elem) != cudaSuccess) return bail(FAM_E_NOMEM);
    cudaMemsetAsync(h->buf[b], 0, h->total * h->elem, h->stream);
  }
  if (cudaMalloc(&h->dinst, sizeof(BatchInst) * n_inst) != cudaSuccess) return bail(FAM_E_NOMEM);
  if (cudaMalloc(&h->ictl, sizeof(BatchCtl) * n_inst) != cudaSuccess) return bail(FAM_E_NOMEM);
  if (cudaMalloc(&h->glob, sizeof(BatchGlobal)) != cudaSuccess) return bail(FAM_E_NOMEM);
  if (cudaMemcpy(h->dinst, h->hinst.data(), sizeof(BatchInst) * n_inst, cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(FAM_E_CUDA);
  if (d == 2) {
    std::vector<Geo> gv(n_inst);
    for (int i = 0; i < n_inst; ++i) {
      const BatchInst& I = h->hinst[i];
      Geo& g = gv[i];
      std::memset(&g, 0, sizeof(g));
      g.nx = I.nx;
      g.ny = I.ny;
      g.px = I.px;
      g.rows = I.rows;
      g.plane = I.plane;
      g.bcx = g.bcy = bc;
      for (int q = 0; q < 4; ++q) g.bc[q] = bc;
      g.dx = I.dx;
      g.dy = I.dy;
      g.idx = I.idx;
      g.idy = I.idy;
      g.nm = 3;
      g.euler = 1;
    }
    if (cudaMalloc(&h->dgeo, sizeof(Geo) * n_inst) != cudaSuccess) return bail(FAM_E_NOMEM);
    if (cudaMemcpy(h->dgeo, gv.data(), sizeof(Geo) * n_inst, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(FAM_E_CUDA);
  }
  if (build_tiles(h) != FAM_OK) return bail(FAM_E_CUDA);
  if (reset_clock(h) != FAM_OK) return bail(FAM_E_CUDA);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(FAM_E_CUDA);
  *out = h;
  return FAM_OK;
}

fam_status fam_batch_create(fam_batch_t* out, int n_inst, const int* nx, const int* k, double x0, double x1,
                            int equation, int bc, double gamma, int precision, void* stream) {
  return create_batch(out, 1, n_inst, nx, nullptr, k, x0, x1, 0.0, 1.0, equation, bc, gamma, precision, stream);
}

fam_status fam_batch2d_create(fam_batch_t* out, int n_inst, const int* nx, const int* ny, const int* k, double x0,
                              double x1, double y0, double y1, int equation, int bc, double gamma, int precision,
                              void* stream) {
  return create_batch(out, 2, n_inst, nx, ny, k, x0, x1, y0, y1, equation, bc, gamma, precision, stream);
}

void fam_batch_destroy(fam_batch_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  for (int b = 0; b < 3; ++b)
    if (h->buf[b]) cudaFree(h->buf[b]);
  if (h->dinst) cudaFree(h->dinst);
  if (h->dgeo) cudaFree(h->dgeo);
  if (h->dtiles) cudaFree(h->dtiles);
  if (h->ictl) cudaFree(h->ictl);
  if (h->glob) cudaFree(h->glob);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

const char* fam_batch_last_error(fam_batch_t h) { return h ? h->err.c_str() : "null handle"; }

fam_status fam_batch_set_option(fam_batch_t h, const char* key, double v) {
  if (!h || !key) return FAM_E_INVAL;
  std::string k(key);
  if (k == "oe_type") {
    if (v != 0.0 && v != 2.0) return bfail(h, FAM_E_INVAL, "oe_type must be 0 or 2");
    h->oe_type = (int)v;
  } else if (k == "gamma_k") {
    for (auto& I : h->hinst) I.gamma_k = v > 0.0 ? v : (I.k <= 4 ? 25.0 : (h->d == 2 ? 15.0 : 12.5));
    FAMB_CUDA(h, cudaMemcpy(h->dinst, h->hinst.data(), sizeof(BatchInst) * h->n, cudaMemcpyHostToDevice));
  } else if (k == "ax") {
    h->ax = v;
  } else if (k == "tile_x") {
    if (h->d != 1) return bfail(h, FAM_E_INVAL, "tile_x applies to 1D batches (2D: tile2d)");
    if (v != 64.0 && v != 128.0 && v != 256.0) return bfail(h, FAM_E_INVAL, "tile_x must be 64, 128 or 256");
    h->tile_x = (int)v;
    h->dt_valid = false;
    return build_tiles(h);
  } else if (k == "tile2d") {
    if (h->d != 2) return bfail(h, FAM_E_INVAL, "tile2d applies to 2D batches");
    if (v != 0.0 && v != 1.0 && v != 2.0) return bfail(h, FAM_E_INVAL, "tile2d must be 0, 1 or 2");
    h->tile2d = (int)v;
    h->dt_valid = false;
    return build_tiles(h);
  } else if (k == "blocks_per_sm") {
    h->blocks_per_sm = (int)v;
  } else if (k == "pp_limiter") {
    if (v != 0.0 && v != 1.0) return bfail(h, FAM_E_INVAL, "pp_limiter must be 0 or 1");
    if (v != 0.0 && (h->d != 1 || h->eq != FAM_EULER))
      return bfail(h, FAM_E_UNSUPPORTED, "pp_limiter is built for 1D Euler batches");
    h->pp = (int)v;
  } else if (k == "wait_limit_ns" || k == "test_barrier_extra") {
    // read by the kernels from the batch's device block at run time: no
    // re-capture, and the step sizes stay valid
    if (k == "wait_limit_ns") {
      if (!(v >= 0.0) || v > 6.0e10) return bfail(h, FAM_E_INVAL, "wait_limit_ns must be in [0, 6e10]");
      h->wait_ns = (unsigned long long)v;
    } else {
      if (v != 0.0 && v != 1.0) return bfail(h, FAM_E_INVAL, "test_barrier_extra must be 0 or 1");
      h->barrier_extra = (unsigned int)v;
    }
    batch_glob_limits<<<1, 1, 0, h->stream>>>(h->glob, h->wait_ns, h->barrier_extra);
    FAMB_CUDA(h, cudaGetLastError());
    FAMB_CUDA(h, cudaStreamSynchronize(h->stream));
    return FAM_OK;
  } else {
    return bfail(h, FAM_E_INVAL, "unknown option " + k);
  }
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  h->dt_valid = false;
  return FAM_OK;
}

static fam_status batch_copy(fam_batch* h, void* dst_user, const void* src_user, int on_device, int b, bool in) {
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : (in ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost);
  long long uoff = 0;
  if (h->d == 2) {
    // per instance and plane: ny rows of nx cells, interior at padded (G, G)
    for (int i = 0; i < h->n; ++i) {
      const BatchInst& I = h->hinst[i];
      const size_t row = (size_t)I.nx * h->elem;
      for (int p = 0; p < h->np; ++p) {
        char* dev = reinterpret_cast<char*>(h->buf[b]) +
                    (size_t)(I.off + (long long)p * I.plane + (long long)G * I.px + G) * h->elem;
        const size_t u = (size_t)(uoff + (long long)p * I.nx * I.ny) * h->elem;
        if (in)
          FAMB_CUDA(h, cudaMemcpy2DAsync(dev, (size_t)I.px * h->elem, reinterpret_cast<const char*>(src_user) + u, row,
                                         row, I.ny, kind, h->stream));
        else
          FAMB_CUDA(h, cudaMemcpy2DAsync(reinterpret_cast<char*>(dst_user) + u, row, dev, (size_t)I.px * h->elem, row,
                                         I.ny, kind, h->stream));
      }
      uoff += (long long)I.nx * I.ny * h->np;
    }
    return FAM_OK;
  }
  for (int i = 0; i < h->n; ++i) {
    const BatchInst& I = h->hinst[i];
    const size_t row = (size_t)I.nx * h->elem;
    char* dev = reinterpret_cast<char*>(h->buf[b]) + (size_t)(I.off + G) * h->elem;
    if (in) {
      const char* src = reinterpret_cast<const char*>(src_user) + uoff * h->elem;
      FAMB_CUDA(h, cudaMemcpy2DAsync(dev, (size_t)I.px * h->elem, src, row, row, h->np, kind, h->stream));
    } else {
      char* dst = reinterpret_cast<char*>(dst_user) + uoff * h->elem;
      FAMB_CUDA(h, cudaMemcpy2DAsync(dst, row, dev, (size_t)I.px * h->elem, row, h->np, kind, h->stream));
    }
    uoff += (long long)I.nx * h->np;
  }
  return FAM_OK;
}

fam_status fam_batch_set_state(fam_batch_t h, const void* U, int on_device) {
  if (!h || !U) return FAM_E_INVAL;
  fam_status s = batch_copy(h, nullptr, U, on_device, 0, true);
  if (s) return s;
  s = fill_ghosts(h, 0);
  if (s) return s;
  s = reset_clock(h);
  if (s) return s;
  FAMB_CUDA(h, cudaStreamSynchronize(h->stream));
  h->have_state = true;
  h->dt_valid = false;
  return FAM_OK;
}

fam_status fam_batch_get_state(fam_batch_t h, void* U, int on_device) {
  if (!h || !U) return FAM_E_INVAL;
  if (!h->have_state) return bfail(h, FAM_E_STATE, "no state");
  fam_status s = batch_copy(h, U, nullptr, on_device, 0, false);
  if (s) return s;
  FAMB_CUDA(h, cudaStreamSynchronize(h->stream));
  return FAM_OK;
}

fam_status fam_batch_run(fam_batch_t h, long nsteps, double cfl) {
  if (!h) return FAM_E_INVAL;
  if (nsteps < 0) return bfail(h, FAM_E_INVAL, "nsteps < 0");
  fam_status s = ensure_init(h, cfl);
  if (s) return s;
  if (nsteps == 0) return FAM_OK;
  for (auto& kv : h->graphs)
    if (kv.first.first == nsteps && kv.first.second == cfl) {
      FAMB_CUDA(h, cudaGraphLaunch(kv.second, h->stream));
      return FAM_OK;
    }
  // capture the persistent cooperative launch into a graph once per (nsteps, cfl)
  cudaGraph_t graph;
  FAMB_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = launch(h, nsteps, cfl, 0);
  cudaError_t ce = cudaStreamEndCapture(h->stream, &graph);
  if (le != cudaSuccess || ce != cudaSuccess) {
    // capture of a cooperative launch not available: launch directly
    if (ce == cudaSuccess) cudaGraphDestroy(graph);
    cudaGetLastError();
    FAMB_CUDA(h, launch(h, nsteps, cfl, 0));
    return FAM_OK;
  }
  cudaGraphExec_t exec;
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    FAMB_CUDA(h, launch(h, nsteps, cfl, 0));
    return FAM_OK;
  }
  h->graphs.push_back({{nsteps, cfl}, exec});
  FAMB_CUDA(h, cudaGraphLaunch(exec, h->stream));
  return FAM_OK;
}

fam_status fam_batch_sync(fam_batch_t h) {
  if (!h) return FAM_E_INVAL;
  BatchGlobal g;
  FAMB_CUDA(h, cudaMemcpyAsync(&g, h->glob, sizeof(g), cudaMemcpyDeviceToHost, h->stream));
  FAMB_CUDA(h, cudaStreamSynchronize(h->stream));
  if (g.status & kStatusTimeout) return bfail(h, FAM_E_TIMEOUT, "grid barrier timed out");
  if (g.status & (kStatusNonFinite | kStatusNonPhysical)) return bfail(h, FAM_E_NONPHYSICAL, "non-physical state");
  return FAM_OK;
}

fam_status fam_batch_times(fam_batch_t h, double* t, double* dt, long* steps) {
  if (!h) return FAM_E_INVAL;
  std::vector<BatchCtl> c(h->n);
  FAMB_CUDA(h, cudaMemcpyAsync(c.data(), h->ictl, sizeof(BatchCtl) * h->n, cudaMemcpyDeviceToHost, h->stream));
  FAMB_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int i = 0; i < h->n; ++i) {
    if (t) t[i] = c[i].t;
    if (dt) dt[i] = c[i].dt;
    if (steps) steps[i] = (long)c[i].steps;
  }
  return FAM_OK;
}

fam_status fam_batch_rejected_steps(fam_batch_t h, unsigned long long* count) {
  if (!h || !count) return FAM_E_INVAL;
  std::vector<BatchCtl> c(h->n);
  FAMB_CUDA(h, cudaMemcpyAsync(c.data(), h->ictl, sizeof(BatchCtl) * h->n, cudaMemcpyDeviceToHost, h->stream));
  FAMB_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int i = 0; i < h->n; ++i) count[i] = c[i].rejected;
  return FAM_OK;
}

fam_status fam_batch_health(fam_batch_t h, unsigned long long* ntrace, int* status, long* bad_step) {
  if (!h) return FAM_E_INVAL;
  std::vector<BatchCtl> c(h->n);
  FAMB_CUDA(h, cudaMemcpyAsync(c.data(), h->ictl, sizeof(BatchCtl) * h->n, cudaMemcpyDeviceToHost, h->stream));
  FAMB_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int i = 0; i < h->n; ++i) {
    if (ntrace) ntrace[i] = c[i].ntrace;
    if (status) status[i] = c[i].status == 0u ? FAM_OK : FAM_E_NONPHYSICAL;
    if (bad_step) bad_step[i] = (long)c[i].bad_step;
  }
  return FAM_OK;
}

fam_status fam_batch_info(fam_batch_t h, int* tile_x, int* grid, long* ntiles, long* cells) {
  if (!h) return FAM_E_INVAL;
  int g = 0;
  FAMB_CUDA(h, launch(h, 0, 1.0, 0, true, &g));
  if (tile_x) *tile_x = h->d == 2 ? kBatchTile2D[h->tile2d][0] : h->tile_x;
  if (grid) *grid = g;
  if (ntiles) *ntiles = h->ntiles;
  if (cells) *cells = h->cells;
  return FAM_OK;
}

fam_status fam_batch_tune(fam_batch_t h, double cfl, int probe_steps, const char* cache_path, int* tile_x_out,
                          int* blocks_per_sm_out) {
  if (!h) return FAM_E_INVAL;
  if (!h->have_state) return bfail(h, FAM_E_STATE, "no state");
  if (probe_steps < 1) probe_steps = 1;
  // key of this configuration
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, dev);
  std::ostringstream key;
  key << prop.name << "|d" << h->d << "|eq" << h->eq << "|p" << h->prec << "|n" << h->n << "|cells" << h->cells
      << (h->pp ? "|pp" : "");
  // candidate tile shapes: 1D tile widths, 2D indices into kBatchTile2D
  auto& shape = h->d == 1 ? h->tile_x : h->tile2d;
  if (cache_path && cache_path[0]) {
    std::ifstream f(cache_path);
    std::string line;
    while (std::getline(f, line)) {
      std::istringstream ls(line);
      std::string k;
      int tx = 0, bps = 0;
      if (std::getline(ls, k, '\t') && (ls >> tx >> bps) && k == key.str()) {
        shape = tx;
        h->blocks_per_sm = bps;
        fam_status s = build_tiles(h);
        if (s) return s;
        h->dt_valid = false;
        if (tile_x_out) *tile_x_out = h->d == 2 ? kBatchTile2D[h->tile2d][0] : h->tile_x;
        if (blocks_per_sm_out) *blocks_per_sm_out = bps;
        return FAM_OK;
      }
    }
  }
  // save the state and the clocks, time each candidate from the same state,
  // restore both
  void* save = nullptr;
  FAMB_CUDA(h, cudaMalloc(&save, h->total * h->elem + sizeof(BatchCtl) * h->n + sizeof(BatchGlobal)));
  BatchCtl* save_ctl = reinterpret_cast<BatchCtl*>(static_cast<char*>(save) + h->total * h->elem);
  BatchGlobal* save_glob = reinterpret_cast<BatchGlobal*>(save_ctl + h->n);
  FAMB_CUDA(h, cudaMemcpyAsync(save, h->buf[0], h->total * h->elem, cudaMemcpyDeviceToDevice, h->stream));
  FAMB_CUDA(h, cudaMemcpyAsync(save_ctl, h->ictl, sizeof(BatchCtl) * h->n, cudaMemcpyDeviceToDevice, h->stream));
  FAMB_CUDA(h, cudaMemcpyAsync(save_glob, h->glob, sizeof(BatchGlobal), cudaMemcpyDeviceToDevice, h->stream));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best_tx = shape, best_b = h->blocks_per_sm;
  float best = 1e30f;
  const int txs1[3] = {64, 128, 256}, txs2[3] = {0, 1, 2};
  for (int tx : (h->d == 1 ? txs1 : txs2)) {
    shape = tx;
    if (build_tiles(h) != FAM_OK) continue;
    int occ_grid = 0;
    h->blocks_per_sm = 0;
    if (launch(h, 0, cfl, 0, true, &occ_grid) != cudaSuccess) continue;
    for (int frac = 1; frac <= 2; ++frac) {
      int dev_sms = prop.multiProcessorCount;
      int occ = std::max(1, occ_grid / dev_sms);
      int bps = frac == 1 ? occ : std::max(1, occ / 2);
      if (frac == 2 && bps == occ) continue;
      h->blocks_per_sm = bps;
      cudaMemcpyAsync(h->buf[0], save, h->total * h->elem, cudaMemcpyDeviceToDevice, h->stream);
      reset_clock(h);
      if (launch(h, 0, cfl, 1) != cudaSuccess) { cudaGetLastError(); continue; }
      cudaEventRecord(e0, h->stream);
      cudaError_t le = launch(h, probe_steps, cfl, 0);
      cudaEventRecord(e1, h->stream);
      if (le != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) { cudaGetLastError(); continue; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_tx = tx;
        best_b = bps;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  shape = best_tx;
  h->blocks_per_sm = best_b;
  fam_status s = build_tiles(h);
  FAMB_CUDA(h, cudaMemcpyAsync(h->buf[0], save, h->total * h->elem, cudaMemcpyDeviceToDevice, h->stream));
  FAMB_CUDA(h, cudaMemcpyAsync(h->ictl, save_ctl, sizeof(BatchCtl) * h->n, cudaMemcpyDeviceToDevice, h->stream));
  FAMB_CUDA(h, cudaMemcpyAsync(h->glob, save_glob, sizeof(BatchGlobal), cudaMemcpyDeviceToDevice, h->stream));
  FAMB_CUDA(h, cudaStreamSynchronize(h->stream));
  cudaFree(save);
  h->dt_valid = false;
  if (s) return s;
  if (cache_path && cache_path[0]) {
    std::ofstream f(cache_path, std::ios::app);
    f << key.str() << '\t' << best_tx << ' ' << best_b << '\n';
  }
  if (tile_x_out) *tile_x_out = h->d == 2 ? kBatchTile2D[h->tile2d][0] : h->tile_x;
  if (blocks_per_sm_out) *blocks_per_sm_out = best_b;
  return FAM_OK;
}

fam_status fam_batch_tile(fam_batch_t h, int* tile_x, int* tile_y) {
  if (!h) return FAM_E_INVAL;
  if (tile_x) *tile_x = h->d == 2 ? kBatchTile2D[h->tile2d][0] : h->tile_x;
  if (tile_y) *tile_y = h->d == 2 ? kBatchTile2D[h->tile2d][1] : 1;
  return FAM_OK;
}

}  // extern "C"
