// fam_batch.cuh -- data shared by the batched persistent kernels (1D in
// fam_batch.cu, 2D in fam_batch2d.cu) and their host code.
#pragma once

#include <cuda_runtime.h>

#include "fam_common.cuh"

namespace fam {

// One instance of a batch: its planes start at element `off` of each packed
// state buffer; plane stride `plane`, row pitch px (padded, G ghost layers).
struct BatchInst {
  long long off;    // element offset of plane 0
  long long plane;  // elements per plane (px * rows)
  int nx, ny, px, rows, k, pad;
  double dx, dy, idx, idy;
  double gamma_k;
};

// Per-instance clock: step size, time, speed maxima of the current step
// (x and y, as bit patterns of non-negative doubles), steps taken; the
// instance's own health: face points whose trace had no spectral radius,
// status bits, and the step whose output was first flagged (0: none; the
// instance stops after that step while the others go on).  BP/PP safeguard
// (1D Euler), step rejection: the stage tiles set bit s of stage_bad when a
// cell average of stage s leaves the admissible set; the instance's later
// stages and its OE then skip the step (A keeps U^n) and the clock pass
// discards it, halves the step size (retry_exp halvings so far, at most 30)
// and counts it in rejected.
struct BatchCtl {
  double dt, t;
  unsigned long long alpha_bits, alpha_bits_y;
  unsigned long long steps;
  unsigned long long ntrace;
  unsigned int status, stage_bad;
  unsigned long long bad_step;
  unsigned int retry_exp, pad;
  unsigned long long rejected;
};

// End of an instance's step in the clock pass: a flagged instance records
// the step and stops (dt = 0); its flags join the batch's status word.
__device__ __forceinline__ void close_instance_step(BatchCtl& c, unsigned int* gstatus) {
  if (c.status != 0u) {
    if (c.bad_step == 0ull) c.bad_step = c.steps;
    c.dt = 0.0;
    atomicOr(gstatus, c.status);
  }
}

// Barrier state and status word of a batch, plus the barrier's wait limit
// (wait_ns, 0: kWaitLimitNs) and a test hook: `extra` arrivals that never
// come are added to the barrier's expected count, so that a test can make
// the bounded wait run out (nothing hangs: every waiter gives up after
// wait_ns and the kernel returns with kStatusTimeout).
struct BatchGlobal {
  unsigned int bar_count, bar_gen, abort, status;
  unsigned int extra, pad;
  unsigned long long wait_ns;
};

// Grid-wide barrier of a cooperative launch, with a bounded wait: a block
// that waits longer than the limit (or sees another block give up) records a
// timeout and returns false so that the whole kernel exits.
__device__ inline bool grid_barrier(BatchGlobal* g, unsigned int nblocks_launched) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vgen = &g->bar_gen;
    volatile unsigned int* vab = &g->abort;
    const unsigned int nblocks = nblocks_launched + g->extra;
    const unsigned long long limit = g->wait_ns != 0ull ? g->wait_ns : kWaitLimitNs;
    const unsigned int my = atomicAdd(&g->bar_gen, 0u);
    __threadfence();
    if (atomicAdd(&g->bar_count, 1u) == nblocks - 1) {
      atomicExch(&g->bar_count, 0u);
      __threadfence();
      atomicAdd(&g->bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*vgen == my) {
        if (*vab) { ok = 0; break; }
        if (global_ns() - t0 > limit) {
          atomicExch(&g->abort, 1u);
          atomicOr(&g->status, kStatusTimeout);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Arguments of one 2D batched launch (fam_batch2d.cu).
struct Batch2DArgs {
  const BatchInst* inst;
  const Geo* geos;    // per-instance geometry (2D)
  const int4* tiles;  // (instance, x0, y0, -)
  int ntiles, ninst;
  void* A;
  void* B;
  void* C;
  BatchCtl* ictl;
  BatchGlobal* glob;
  int equation;
  double gamma;
  int nsteps;
  double cfl;
  int oe_type, bc, init;
};

}  // namespace fam

// 2D batched persistent launch, one per precision (fam_batch2d.cu compiled
// with FAM_P = 64 / 32).  tile2d indexes the tile shapes (32x8, 32x4, 16x8);
// blocks_per_sm <= 0 takes the occupancy maximum.  With query_only, only
// *grid_out is computed.
cudaError_t fam_batch2d_launch_p64(const fam::Batch2DArgs& a, int tile2d, int blocks_per_sm, bool query_only,
                                   int* grid_out, cudaStream_t stream);
cudaError_t fam_batch2d_launch_p32(const fam::Batch2DArgs& a, int tile2d, int blocks_per_sm, bool query_only,
                                   int* grid_out, cudaStream_t stream);
