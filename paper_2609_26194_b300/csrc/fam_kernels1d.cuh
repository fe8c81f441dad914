// fam_kernels1d.cuh -- 1D FAM kernels (sm_103a).
//
//  stage1d  one SSP-RK3 stage (eq. 3 with the Shu--Osher coefficients of
//           eq. 12): TMA-staged tile + halo of the moment planes, compact
//           reconstruction (eq. 5 / 6), Rusanov flux at every face, 4-point
//           Gauss volume term, residual of eq. (1dSemi), combination, ghosts.
//  oe1d     end-of-step OE (eq. 9 / eq. 1dOE_system, Tab. sigma1d) fused with
//           the max Rusanov speed for the next step.
//  alpha1d  the speed reduction alone (first step).
#pragma once

#include "fam_kernels2d.cuh"
#include "fam_pp.cuh"

namespace fam {

template <typename T, int NC, int TX>
struct Smem1D {
  static constexpr int NP = NC * 2;
  static constexpr int HX = TX + 4;
  static constexpr int TILE = NP * HX;
  static constexpr size_t bytes_stage = sizeof(T) * (size_t)(TILE + 2 * (TX + 1) * NC) + 16 + 64 * sizeof(double);
  static constexpr size_t bytes_oe = sizeof(T) * (size_t)(TILE + 2 * (TX + 2) * NC + (TX + 2)) + 16 + 64 * sizeof(double);
};

template <typename T, int NP, int HX>
__device__ __forceinline__ bool load_tile_1d(T* tile, uint64_t* bar, const CUtensorMap* tm, int x0, FamCtl* ctl) {
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, (uint32_t)(sizeof(T) * NP * HX));
    tma_load_2d(tile, tm, bar, x0, 0);
  }
  bool ok = mbar_wait(bar, 0);
  if (!ok) {
    atomicOr(&ctl->status, kStatusTimeout);
    mbar_wait(bar, 0);
  }
  return ok;
}

template <typename T, int K, int HX>
__device__ __forceinline__ void coef1d(const T* tile, int c, int hx, T* cf) {
  const T* pa = tile + (size_t)(c * 2) * HX;
  const T* pm = tile + (size_t)(c * 2 + 1) * HX;
  Recon1D<K>::coef(pa[hx - 1], pa[hx], pa[hx + 1], pm[hx - 1], pm[hx], pm[hx + 1], cf);
}

// One stage on a tile already staged in shared memory: tile = the NP planes
// of cells x0-2 .. x0+TX+1 (padded columns x0 .. x0+TX+3).  U0 / Uout point
// at the instance's plane 0.  Called by all TX threads of the block.
// ntrace (may be null) accumulates the faces of this tile at which a trace
// has no spectral radius; each face of the grid is counted by one tile only.
// PP (a physics with a safeguard, PH::kLimiter != 0): the stage's
// reconstructions are scaled by it (fam_pp.cuh) before any evaluation.
template <typename T, int K, class PH, int TX, bool PP = false>
__device__ __forceinline__ void stage1d_tile(const T* tile, T* fL, T* fR, const T* __restrict__ U0,
                                             T* __restrict__ Uout, const Geo& geo, const PH& ph, const T dt,
                                             const int stage, const int x0, unsigned long long* ntrace,
                                             unsigned int* stage_bad = nullptr) {
  constexpr int NC = PH::NC;
  constexpr int HX = TX + 4;
  constexpr int D = K - 1;
  const int tx = threadIdx.x, hx = tx + 2;
  const T wg[4] = {T(famgen::kGaussW[0]), T(famgen::kGaussW[1]), T(famgen::kGaussW[2]), T(famgen::kGaussW[3])};
  T VA[PH::NVA];
#pragma unroll
  for (int q = 0; q < PH::NVA; ++q) VA[q] = T(0);
  T uq[NC][4];
  if constexpr (PP && PH::kLimiter != 0) {
    T cfa[NC][K];
#pragma unroll
    for (int c = 0; c < NC; ++c) coef1d<T, K, HX>(tile, c, hx, cfa[c]);
    pp_limit_any_1d<T, K, PH>(cfa, ph);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      sym_pair<T, D, kRowInner>(cfa[c], uq[c][2], uq[c][1]);
      sym_pair<T, D, kRowOuter>(cfa[c], uq[c][3], uq[c][0]);
      T r, l;
      sym_pair<T, D, kRowHalf>(cfa[c], r, l);
      fL[(tx + 1) * NC + c] = r;
      fR[tx * NC + c] = l;
    }
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T cf[K];
      coef1d<T, K, HX>(tile, c, hx, cf);
      sym_pair<T, D, kRowInner>(cf, uq[c][2], uq[c][1]);
      sym_pair<T, D, kRowOuter>(cf, uq[c][3], uq[c][0]);
      T r, l;
      sym_pair<T, D, kRowHalf>(cf, r, l);
      fL[(tx + 1) * NC + c] = r;
      fR[tx * NC + c] = l;
    }
  }
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    T u[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) u[c] = uq[c][g];
    ph.vol_acc(u, wg[g], VA);
  }
  // ring: cell x0-1 (right trace -> face 0) and cell x0+TX (left trace -> face TX)
  if (tx < 2) {
    const int rh = tx == 0 ? 1 : TX + 2;
    if constexpr (PP && PH::kLimiter != 0) {
      T cfa[NC][K];
#pragma unroll
      for (int c = 0; c < NC; ++c) coef1d<T, K, HX>(tile, c, rh, cfa[c]);
      pp_limit_any_1d<T, K, PH>(cfa, ph);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        T r, l;
        sym_pair<T, D, kRowHalf>(cfa[c], r, l);
        if (tx == 0) fL[c] = r;
        else fR[TX * NC + c] = l;
      }
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        T cf[K], r, l;
        coef1d<T, K, HX>(tile, c, rh, cf);
        sym_pair<T, D, kRowHalf>(cf, r, l);
        if (tx == 0) fL[c] = r;
        else fR[TX * NC + c] = l;
      }
    }
  }
  __syncthreads();
  unsigned nbad = 0;
  for (int f = tx; f <= TX; f += TX) {
    T uL[NC], uR[NC], FL[NC], FR[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) { uL[c] = fL[f * NC + c]; uR[c] = fR[f * NC + c]; }
    const T sL = ph.flux_x(uL, FL), sR = ph.flux_x(uR, FR);
    const T a = rusanov_speed(sL, sR);
#pragma unroll
    for (int c = 0; c < NC; ++c) fL[f * NC + c] = T(0.5) * (FL[c] + FR[c]) - T(0.5) * a * (uR[c] - uL[c]);
    // owner: the tile of the face's right cell (the grid's last face: its left cell's)
    if ((nan_bits(sL) || nan_bits(sR)) && x0 + f <= geo.nx && (f < TX || x0 + f == geo.nx)) ++nbad;
  }
  warp_count_add(ntrace, nbad);
  __syncthreads();
  const int i = x0 + tx;
  if (i >= geo.nx) return;  // no barrier follows
  const T idx_ = T(geo.idx);
  T avg[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) avg[c] = tile[(size_t)(c * 2) * HX + hx];
  T V1[NC];
  ph.vol_finish(VA, avg, V1);
  T w0, w1;
  stage_weights<T>(stage, w0, w1);
  T vout[NC];  // this cell's output averages (the safeguard's stage check)
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const T fl = fL[tx * NC + c], fr = fL[(tx + 1) * NC + c];
    T R[2];
    R[0] = -(fr - fl) * idx_;
    R[1] = (V1[c] - T(0.5) * (fr + fl)) * idx_;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const int p = c * 2 + m;
      T v;
      if (stage == 0) {
        v = R[m];
      } else {
        const T us = tile[(size_t)p * HX + hx];
        if (stage == 1) {
          v = us + dt * R[m];
        } else {
          const T u0 = U0[cell_index(geo, p, 0, i)];
          v = w0 * u0 + w1 * (us + dt * R[m]);
        }
      }
      if (m == 0) vout[c] = v;
      store_with_ghosts(Uout, geo, p, 0, i, v);
    }
  }
  // BP/PP safeguard: a stage output average outside the admissible set
  // discards the step (the OE then writes nothing; see FamCtl::stage_bad);
  // bit `stage` records which stage it was
  if (stage_bad != nullptr && stage != 0 && !ph.admissible(vout)) atomicOr(stage_bad, 1u << stage);
}


template <typename T, int K, class PH, int TX, bool PP = false>
__global__ void __launch_bounds__(TX)
    stage1d(const __grid_constant__ CUtensorMap tm_in, const T* __restrict__ U0, T* __restrict__ Uout,
            const Geo geo, const PH ph, FamCtl* __restrict__ ctl, const int stage) {
  constexpr int NC = PH::NC;
  using S = Smem1D<T, NC, TX>;
  constexpr int NP = S::NP, HX = S::HX;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  T* fL = tile + S::TILE;          // left-side trace at face f (0..TX), later the flux
  T* fR = fL + (TX + 1) * NC;      // right-side trace at face f
  uint64_t* bar = reinterpret_cast<uint64_t*>(fR + (TX + 1) * NC);

  const double dtd = (stage == 0) ? 0.0 : ctl->dt;
  if (stage != 0 && !pos_bits(dtd)) return;
  if (PP && stage >= 2 && ctl->stage_bad != 0u) return;  // an earlier stage discarded the step
  const int x0 = blockIdx.x * TX;
  if (threadIdx.x == 0) prefetch_tmap(&tm_in);
  if (!load_tile_1d<T, NP, HX>(tile, bar, &tm_in, x0, ctl)) return;
  stage1d_tile<T, K, PH, TX, PP>(tile, fL, fR, U0, Uout, geo, ph, T(dtd), stage, x0, &ctl->ntrace,
                                 PP ? &ctl->stage_bad : nullptr);
}

// OE on a staged tile (layout as for stage1d_tile); returns this thread's
// cell speed (0 outside the grid) for the CFL reduction.
template <typename T, int K, class PH, int TX>
__device__ __forceinline__ T oe1d_tile(const T* tile, T* tr, T* sp, T* __restrict__ Uout, const Geo& geo,
                                            const PH& ph, const T dt, const int oe_type, const T gamma_k,
                                            const int x0, unsigned int* status, const FamCtl* ctl = nullptr) {
  constexpr int NC = PH::NC;
  constexpr int HX = TX + 4;
  constexpr int D = K - 1;
  constexpr int RX = TX + 2;
  for (int q = threadIdx.x; q < RX; q += TX) {
    const int hx = q + 1;  // ring coordinate q <-> cell x0 + q - 1
    T u[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      T cf[K], r, l;
      coef1d<T, K, HX>(tile, c, hx, cf);
      sym_pair<T, D, kRowHalf>(cf, r, l);
      tr[(q * 2 + 0) * NC + c] = l;
      tr[(q * 2 + 1) * NC + c] = r;
      u[c] = tile[(size_t)(c * 2) * HX + hx];
    }
    sp[q] = ph.speed_x(u);
  }
  __syncthreads();
  const int tx = threadIdx.x, i = x0 + tx;
  T my_speed = T(0);
  if (i < geo.nx) {
    const int q = tx + 1, hx = tx + 2;
    T sig = T(0);
    T uavg[NC];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const T jl = tr[(q * 2 + 0) * NC + c] - tr[((q - 1) * 2 + 1) * NC + c];
      const T jr = tr[((q + 1) * 2 + 0) * NC + c] - tr[(q * 2 + 1) * NC + c];
      const T* pa = tile + (size_t)(c * 2) * HX;
      const T vm = pa[hx - 1], v0 = pa[hx], vp = pa[hx + 1];
      T Dn, eps;
      if (oe_type == 1) {
        Dn = T(__longlong_as_double((long long)ctl->t1_dev_bits[c]));
        eps = T(1e-14) * max_nonneg(T(__longlong_as_double((long long)ctl->t1_maxabs_bits[c])), T(1));
      } else {
        // maxima of non-negative values on their bit patterns (integer pipes)
        const T S = vm + v0 + vp;
        Dn = max_nonneg(max_nonneg(abs_bits(vm - S), abs_bits(v0 - S)), abs_bits(vp - S));
        eps = T(1e-14) * max_nonneg(max_nonneg(max_nonneg(abs_bits(vm), abs_bits(v0)), abs_bits(vp)), T(1));
      }
      if (oe_type != 0 && !less_nonneg(Dn, eps))
        sig = max_nonneg(sig, gamma_k * (fabs(jl) + fabs(jr)) * Fast<T>::rcp(Dn));
    }
    const T beta = max_nonneg(max_nonneg(sp[q - 1], sp[q]), sp[q + 1]);
    const T theta = beta * dt * sig * T(geo.idx);
    const T delta = Fast<T>::exp_(-theta);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const T a = tile[(size_t)(c * 2) * HX + hx];
      const T m = tile[(size_t)(c * 2 + 1) * HX + hx] * delta;
      uavg[c] = a;
      if (!finite_bits(a) || !finite_bits(m)) ok = false;
      store_with_ghosts(Uout, geo, c * 2 + 0, 0, i, a);
      store_with_ghosts(Uout, geo, c * 2 + 1, 0, i, m);
    }
    if (!ok) atomicOr(status, kStatusNonFinite);
    else if (!ph.admissible(uavg)) atomicOr(status, kStatusNonPhysical);
    my_speed = sp[q];
  }
  return my_speed;
}

template <typename T, int K, class PH, int TX>
__global__ void __launch_bounds__(TX)
    oe1d(const __grid_constant__ CUtensorMap tm_in, T* __restrict__ Uout, const Geo geo, const PH ph,
         FamCtl* __restrict__ ctl, const int oe_type, const T gamma_k, const double dt_override) {
  constexpr int NC = PH::NC;
  using S = Smem1D<T, NC, TX>;
  constexpr int NP = S::NP, HX = S::HX;
  constexpr int RX = TX + 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  T* tr = tile + S::TILE;          // traces [RX][2][NC]: (-1/2, +1/2)
  T* sp = tr + 2 * RX * NC;        // speeds at averages [RX]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sp + RX);
  double* red = reinterpret_cast<double*>(bar + 2);

  const bool reduce = !nonneg_bits(dt_override);
  const double dtd = reduce ? ctl->dt : dt_override;
  if (!pos_bits(dtd) && reduce) return;
  if (reduce && ctl->stage_bad != 0u) {  // the step is discarded: U^n stays in Uout
    if (threadIdx.x == 0) step_epilogue(ctl, gridDim.x, true);
    return;
  }
  const int x0 = blockIdx.x * TX;
  if (threadIdx.x == 0) prefetch_tmap(&tm_in);
  if (!load_tile_1d<T, NP, HX>(tile, bar, &tm_in, x0, ctl)) return;
  const T my_speed =
      oe1d_tile<T, K, PH, TX>(tile, tr, sp, Uout, geo, ph, T(dtd), oe_type, gamma_k, x0, &ctl->status, ctl);
  if (!reduce) return;
  const T mx = block_max<TX>(my_speed, red);
  if (threadIdx.x == 0) {
    atomic_max_nonneg(&ctl->alpha_bits[0], (double)mx);
    step_epilogue(ctl, gridDim.x, true);
  }
}

// ---------------------------------------------------------------------------
// Type-I OE denominators (Tab. sigma1d / sigma2d): grid mean, max |u| and
// D_Omega = max |u - mean| of the cell averages per component.  The sum is
// deterministic: fixed-order block partials, summed in order by one block.
// ---------------------------------------------------------------------------
template <typename T, int NT>
__global__ void __launch_bounds__(NT) typeI_partial(const T* __restrict__ U, const Geo geo, int nc, int nm,
                                                    double* __restrict__ partial, FamCtl* __restrict__ ctl) {
  __shared__ double sh[NT];
  const long long n = (long long)geo.nx * geo.ny;
  for (int c = 0; c < nc; ++c) {
    double s = 0.0, mabs = 0.0;
    for (long long q = blockIdx.x * (long long)NT + threadIdx.x; q < n; q += (long long)gridDim.x * NT) {
      const int i = (int)(q % geo.nx), j = (int)(q / geo.nx);
      const double v = (double)U[cell_index(geo, c * nm, j, i)];
      s += v;
      mabs = fmax(mabs, fabs(v));
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[(long long)c * gridDim.x + blockIdx.x] = sh[0];
    __syncthreads();
    const double m = block_max<NT>(mabs, sh);
    if (threadIdx.x == 0) atomic_max_nonneg(&ctl->t1_maxabs_bits[c], m);
    __syncthreads();
  }
}

template <int UNUSED = 0>
__global__ void typeI_final(const double* __restrict__ partial, int nblocks, int nc, long long ncells,
                            FamCtl* __restrict__ ctl) {
  if (threadIdx.x < nc) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[(long long)threadIdx.x * nblocks + b];
    ctl->t1_mean[threadIdx.x] = s / (double)ncells;
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) typeI_dev(const T* __restrict__ U, const Geo geo, int nc, int nm,
                                                FamCtl* __restrict__ ctl) {
  __shared__ double red[64];
  const long long n = (long long)geo.nx * geo.ny;
  for (int c = 0; c < nc; ++c) {
    const double mean = ctl->t1_mean[c];
    double d = 0.0;
    for (long long q = blockIdx.x * (long long)NT + threadIdx.x; q < n; q += (long long)gridDim.x * NT) {
      const int i = (int)(q % geo.nx), j = (int)(q / geo.nx);
      d = fmax(d, fabs((double)U[cell_index(geo, c * nm, j, i)] - mean));
    }
    d = block_max<NT>(d, red);
    if (threadIdx.x == 0) atomic_max_nonneg(&ctl->t1_dev_bits[c], d);
    __syncthreads();
  }
}

template <typename T, class PH, int NT>
__global__ void __launch_bounds__(NT) alpha1d(const T* __restrict__ U, const Geo geo, const PH ph,
                                              FamCtl* __restrict__ ctl) {
  __shared__ double red[64];
  double mx = 0.0;
  for (int i = blockIdx.x * NT + threadIdx.x; i < geo.nx; i += gridDim.x * NT) {
    T u[PH::NC];
#pragma unroll
    for (int c = 0; c < PH::NC; ++c) u[c] = U[cell_index(geo, c * 2, 0, i)];
    mx = fmax(mx, (double)ph.speed_x(u));
  }
  mx = block_max<NT>(mx, red);
  if (threadIdx.x == 0) {
    atomic_max_nonneg(&ctl->alpha_bits[0], mx);
    step_epilogue(ctl, gridDim.x, false);
  }
}

// Safeguard (Euler, Buckley-Leverett): the largest spectral radius at the check points of
// every cell's limited reconstruction of U -> ctl->dt (no time advance); the
// CFL rule of the safeguard (fam_pp.cuh).
template <typename T, int K, class PH, int NT>
__global__ void __launch_bounds__(NT) pp_alpha1d(const T* __restrict__ U, const Geo geo, const PH ph,
                                                  FamCtl* __restrict__ ctl) {
  constexpr int NC = PH::NC, D = K - 1;
  __shared__ double red[64];
  T mx = T(0);
  for (int i = blockIdx.x * NT + threadIdx.x; i < geo.nx; i += gridDim.x * NT) {
    T cf[NC][K];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const T* pa = U + cell_index(geo, c * 2, 0, i);
      const T* pm = U + cell_index(geo, c * 2 + 1, 0, i);
      Recon1D<K>::coef(pa[-1], pa[0], pa[1], pm[-1], pm[0], pm[1], cf[c]);
    }
    T avg[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) avg[c] = cf[c][0];
    pp_limit_any_1d<T, K, PH>(cf, ph);
    mx = max_nonneg(mx, ph.speed_x(avg));
    pp_points_1d<T, K, NC>(cf, [&](const T* u) { mx = max_nonneg(mx, ph.speed_x(u)); });
  }
  const double m = (double)block_max<NT>(mx, red);
  if (threadIdx.x == 0) {
    atomic_max_nonneg(&ctl->alpha_bits[0], m);
    step_epilogue(ctl, gridDim.x, false);
  }
}

}  // namespace fam
