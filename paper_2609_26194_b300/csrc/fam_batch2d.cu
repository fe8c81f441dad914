// fam_batch2d.cu -- many independent 2D FAM problems in one persistent launch.
//
// Compiled once per precision (-DFAM_P=64 / 32).  Instances of uneven grid
// size (nx_i x ny_i) and order k_i (3..6) share the three packed state
// buffers of the batch handle (fam_batch.cu).  Their cells are cut into
// tiles of TX x TY cells; one cooperative persistent kernel walks the tile
// list for each pass of a time step -- stage 1, 2, 3 (eq. 12) and OE
// (eq. 2dOE_sol / 2dOE_system) -- with a bounded grid barrier between
// passes, and a per-instance step-size pass (Sec. 4 CFL rule with the
// instance's own maximum Rusanov speeds) after each step.  The per-tile
// arithmetic is the single-problem device code (stage2d_tile, oe2d_tile),
// so an instance evolves bit for bit as the single-problem kernels with the
// same tile shape evolve it.  Tiles are staged with 16-byte vector loads
// (load_tile_vec; the instances' tensor maps would differ per tile).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/fam.h"
#include "fam_batch.cuh"
#include "fam_kernels2d.cuh"

#ifndef FAM_P
#error "FAM_P must be defined"
#endif

using namespace fam;

namespace {

#if FAM_P == 64
typedef double Real;
#else
typedef float Real;
#endif

template <typename T, class PH, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, stage_min_blocks<T, TX * TY>())
    batched2d_run(const BatchInst* __restrict__ inst, const Geo* __restrict__ geos, const int4* __restrict__ tiles,
                  int ntiles, int ninst, T* A, T* B, T* C, BatchCtl* ictl, BatchGlobal* g, const PH ph, int nsteps,
                  double cfl, int oe_type, int bc, int init) {
  constexpr int NC = PH::NC;
  using S = Smem2D<T, NC, TX, TY>;
  constexpr int NP = S::NP, HX = S::HX, HY = S::HY;
  constexpr int NT = TX * TY;
  constexpr int RX = TX + 2, RY = TY + 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  // stage slots (Smem2D layout; the U^n region is unused: U^n is read from global memory)
  T* xL = tile + S::U0OFF + S::U0T;
  T* xR = xL + S::XF;
  T* yB = xR + S::XF;
  T* yT = yB + S::YF;
  // OE scratch
  T* fc = tile + S::TILE;
  T* sp = fc + 4 * NC * RX * RY;
  __shared__ double red[64];
  const unsigned int nb = gridDim.x;

  if (init) {
    // speeds at the cell averages of A -> first step size of every instance
    for (int t = blockIdx.x; t < ntiles; t += nb) {
      const int4 td = tiles[t];
      const BatchInst I = inst[td.x];
      const int i = td.y + threadIdx.x % TX, j = td.z + threadIdx.x / TX;
      double mx = 0.0, my = 0.0;
      if (i < I.nx && j < I.ny) {
        T u[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c)
          u[c] = A[I.off + (long long)(c * 3) * I.plane + (long long)(j + G) * I.px + (i + G)];
        T sx, sy;
        ph.speeds(u, sx, sy);
        mx = (double)sx;
        my = (double)sy;
      }
      mx = block_max<NT>(mx, red);
      my = block_max<NT>(my, red + 32);
      if (threadIdx.x == 0) {
        atomic_max_nonneg(&ictl[td.x].alpha_bits, mx);
        atomic_max_nonneg(&ictl[td.x].alpha_bits_y, my);
      }
    }
    if (!grid_barrier(g, nb)) return;
    for (int i = blockIdx.x * NT + threadIdx.x; i < ninst; i += nb * NT) {
      const double ax = __longlong_as_double((long long)ictl[i].alpha_bits);
      const double ay = __longlong_as_double((long long)ictl[i].alpha_bits_y);
      double dt = cfl / (ax / inst[i].dx + ay / inst[i].dy);
      if (!(dt > 0.0) || !isfinite(dt)) {
        dt = 0.0;
        ictl[i].status |= kStatusNonFinite;
        atomicOr(&g->status, kStatusNonFinite);
      }
      ictl[i].dt = dt;
      ictl[i].alpha_bits = 0ull;
      ictl[i].alpha_bits_y = 0ull;
    }
    if (!grid_barrier(g, nb)) return;
  }

  for (int s = 0; s < nsteps; ++s) {
    for (int pass = 1; pass <= 4; ++pass) {
      const T* in = pass == 1 ? A : pass == 2 ? B : pass == 3 ? C : B;
      T* out = pass == 1 ? B : pass == 2 ? C : pass == 3 ? B : A;
      for (int t = blockIdx.x; t < ntiles; t += nb) {
        const int4 td = tiles[t];
        const double dtd = ictl[td.x].dt;
        if (!(dtd > 0.0)) continue;
        const BatchInst& I = inst[td.x];
        // the instance's geometry stays in (cached) global memory rather than in registers
        const Geo& geo = geos[td.x];
        __syncthreads();
        load_tile_vec<T, NP, TX, TY, NT>(tile, in + I.off, geo, td.y, td.z);
        __syncthreads();
        T* Uo = out + I.off;
        if (pass < 4) {
          const U0FromGlobal<T> u0src{A + I.off};
          const T dt = T(dtd);
          switch (I.k) {
            case 3: stage2d_tile<T, 3, PH, TX, TY>(tile, xL, xR, yB, yT, Uo, geo, ph, pass, dt, td.y, td.z, u0src, &ictl[td.x].ntrace, T(geo.idx), T(geo.idy)); break;
            case 4: stage2d_tile<T, 4, PH, TX, TY>(tile, xL, xR, yB, yT, Uo, geo, ph, pass, dt, td.y, td.z, u0src, &ictl[td.x].ntrace, T(geo.idx), T(geo.idy)); break;
            case 5: stage2d_tile<T, 5, PH, TX, TY>(tile, xL, xR, yB, yT, Uo, geo, ph, pass, dt, td.y, td.z, u0src, &ictl[td.x].ntrace, T(geo.idx), T(geo.idy)); break;
            default: stage2d_tile<T, 6, PH, TX, TY>(tile, xL, xR, yB, yT, Uo, geo, ph, pass, dt, td.y, td.z, u0src, &ictl[td.x].ntrace, T(geo.idx), T(geo.idy)); break;
          }
        } else {
          const T dt_idx = T(dtd * I.idx), dt_idy = T(dtd * I.idy);
          const T gk = T(I.gamma_k);
          T mx, my;
          switch (I.k) {
            case 3: oe2d_tile<T, 3, PH, TX, TY>(tile, fc, sp, Uo, geo, ph, oe_type, gk, 1, dt_idx, dt_idy, td.y, td.z, nullptr, &ictl[td.x].status, mx, my); break;
            case 4: oe2d_tile<T, 4, PH, TX, TY>(tile, fc, sp, Uo, geo, ph, oe_type, gk, 1, dt_idx, dt_idy, td.y, td.z, nullptr, &ictl[td.x].status, mx, my); break;
            case 5: oe2d_tile<T, 5, PH, TX, TY>(tile, fc, sp, Uo, geo, ph, oe_type, gk, 1, dt_idx, dt_idy, td.y, td.z, nullptr, &ictl[td.x].status, mx, my); break;
            default: oe2d_tile<T, 6, PH, TX, TY>(tile, fc, sp, Uo, geo, ph, oe_type, gk, 1, dt_idx, dt_idy, td.y, td.z, nullptr, &ictl[td.x].status, mx, my); break;
          }
          mx = block_max<NT>(mx, red);
          my = block_max<NT>(my, red + 32);
          if (threadIdx.x == 0) {
            atomic_max_nonneg(&ictl[td.x].alpha_bits, (double)mx);
            atomic_max_nonneg(&ictl[td.x].alpha_bits_y, (double)my);
          }
        }
      }
      if (!grid_barrier(g, nb)) return;
    }
    // per-instance clock and next step size (the single-problem rule of step_epilogue)
    for (int i = blockIdx.x * NT + threadIdx.x; i < ninst; i += nb * NT) {
      BatchCtl c = ictl[i];
      if (c.dt > 0.0) {
        c.t += c.dt;
        c.steps += 1;
        const double ax = __longlong_as_double((long long)c.alpha_bits);
        const double ay = __longlong_as_double((long long)c.alpha_bits_y);
        double dt = cfl / (ax / inst[i].dx + ay / inst[i].dy);
        if (!(dt > 0.0) || !isfinite(dt)) { dt = 0.0; c.status |= kStatusNonFinite; }
        c.dt = dt;
        close_instance_step(c, &g->status);
      }
      c.alpha_bits = 0ull;
      c.alpha_bits_y = 0ull;
      ictl[i] = c;
    }
    if (!grid_barrier(g, nb)) return;
  }
}

template <class PH, int TX, int TY>
cudaError_t launch_shape(const Batch2DArgs& a, const PH& ph, int blocks_per_sm, bool query_only, int* grid_out,
                         cudaStream_t stream) {
  using S = Smem2D<Real, PH::NC, TX, TY>;
  auto fn = batched2d_run<Real, PH, TX, TY>;
  const size_t smem = std::max(S::bytes_stage, S::bytes_oe);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, TX * TY, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorLaunchOutOfResources;
  const int per_sm = blocks_per_sm > 0 ? std::min(blocks_per_sm, occ) : occ;
  const int grid = std::max(1, std::min(sms * per_sm, a.ntiles));
  if (grid_out) *grid_out = grid;
  if (query_only) return cudaSuccess;
  Real* A = reinterpret_cast<Real*>(a.A);
  Real* B = reinterpret_cast<Real*>(a.B);
  Real* C = reinterpret_cast<Real*>(a.C);
  const BatchInst* di = a.inst;
  const Geo* dg = a.geos;
  const int4* dtl = a.tiles;
  int ntiles = a.ntiles, ninst = a.ninst, ns = a.nsteps, oe = a.oe_type, bc = a.bc, init = a.init;
  double cfl = a.cfl;
  BatchCtl* ic = a.ictl;
  BatchGlobal* gl = a.glob;
  void* args[] = {(void*)&di, (void*)&dg, (void*)&dtl, (void*)&ntiles, (void*)&ninst, (void*)&A, (void*)&B, (void*)&C,
                  (void*)&ic, (void*)&gl, (void*)&ph, (void*)&ns, (void*)&cfl, (void*)&oe, (void*)&bc,
                  (void*)&init};
  return cudaLaunchCooperativeKernel((void*)fn, dim3(grid), dim3(TX * TY), args, smem, stream);
}

template <class PH>
cudaError_t launch_tile(const Batch2DArgs& a, const PH& ph, int tile2d, int bps, bool q, int* g, cudaStream_t st) {
  switch (tile2d) {
    case 1: return launch_shape<PH, 32, 4>(a, ph, bps, q, g, st);
    case 2: return launch_shape<PH, 16, 8>(a, ph, bps, q, g, st);
    default: return launch_shape<PH, 32, 8>(a, ph, bps, q, g, st);
  }
}

}  // namespace

#if FAM_P == 64
cudaError_t fam_batch2d_launch_p64(const Batch2DArgs& a, int tile2d, int blocks_per_sm, bool query_only,
                                   int* grid_out, cudaStream_t stream)
#else
cudaError_t fam_batch2d_launch_p32(const Batch2DArgs& a, int tile2d, int blocks_per_sm, bool query_only,
                                   int* grid_out, cudaStream_t stream)
#endif
{
  if (a.equation != FAM_EULER) return cudaErrorInvalidValue;  // the 2D batch is built for the Euler equations
  const Real gm = Real(a.gamma);
  const Euler2D<Real> ph{gm, Real(a.gamma - 1.0), Real(0.5 * (a.gamma - 1.0))};
  return launch_tile(a, ph, tile2d, blocks_per_sm, query_only, grid_out, stream);
}
