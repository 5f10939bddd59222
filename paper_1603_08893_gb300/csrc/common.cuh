// Shared device helpers: complex arithmetic, deterministic block reductions,
// the device-resident solver state and material views.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define RVE_DEV __device__ __forceinline__

// aligned to its size, so that a complex value moves in one vector load or
// store (8 bytes float, 16 bytes double and float-float)
template <typename R>
struct alignas(2 * sizeof(R)) cplx {
  R x, y;
};

template <typename R>
RVE_DEV cplx<R> c_add(cplx<R> a, cplx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R>
RVE_DEV cplx<R> c_sub(cplx<R> a, cplx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <typename R>
RVE_DEV cplx<R> c_mul(cplx<R> a, cplx<R> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename R>
RVE_DEV cplx<R> c_mulc(cplx<R> a, cplx<R> b) {
  return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}

// ---------------------------------------------------------------------------
// Device-resident CG / Newton scalars.  All reductions are FP64.  The fields
// are written only by the single "last block" of a reducing kernel, so every
// kernel that follows in stream order sees them.
// ---------------------------------------------------------------------------
// Status codes mirrored from the public header.
#define RVE_DEV_ERR_CG_MAXIT (-4)
#define RVE_DEV_ERR_CG_BREAKDOWN (-5)
#define RVE_DEV_ERR_NONFINITE (-7)
#define RVE_DEV_ERR_TIMEOUT (-9)

struct SolverState {
  // CG
  double rr;       // r.r of the current iterate
  double bb;       // ||b||^2 of the right-hand side
  double tol2;     // max(eta^2 bb, atol^2)
  double alpha, beta, pAp;
  int it;          // completed CG iterations
  int maxit;
  int done;        // 1: CG finished (converged, failed or bb == 0)
  int status;      // 0 ok, else an RVE_ERR_* code
  double cg_tol, cg_atol;
  double rr_min;    // smallest r.r so far (stagnation test)
  int it_min;       // iteration of rr_min
  int stag;         // > 0: stop after this many iterations without a 10% drop of ||r||
  // Newton
  double dFbar[9];  // macroscopic increment F-bar - <F>
  double Fbar[9];
  double meanX[9];  // <dF> of the CG solution
  double Fn2;       // ||F||^2 after adding the macroscopic increment
  double dF2;       // ||dF||^2 of the last Newton update
  double Pbar[9];
  double meanF[9];
  double adjW[9];   // W / n of the adjoint right-hand side G : (K : W) / n
  double Kmean[9];  // <K : (U + x)> of the homogenised-tangent column
  int err_flags;    // bit 0: det F <= 0, bit 1: non-finite value
  int dev_timeout;  // set by a thread block whose bounded wait on its own copies gave up
  // reduction counters (one per reducing kernel family)
  unsigned int counter[8];
};

enum ReduceSlot {
  SLOT_PAP = 0,
  SLOT_RR = 1,
  SLOT_BB = 2,
  SLOT_MEAN = 3,
  SLOT_NORM = 4,
  SLOT_MISC = 5,
};


// CG bookkeeping once r.r of the new residual is known (one thread):
// iteration count, convergence, stagnation (float32 CG), iteration limit,
// beta = rr_new / rr.
RVE_DEV void cg_after_rr(SolverState* st, double rr_new) {
  st->it += 1;
  if (!isfinite(rr_new)) {
    st->status = RVE_DEV_ERR_NONFINITE;
    st->done = 1;
  } else if (rr_new <= st->tol2) {
    st->rr = rr_new;
    st->done = 1;
  } else if (st->stag > 0 && rr_new >= 0.81 * st->rr_min && st->it - st->it_min >= st->stag) {
    // no 10% decrease of ||r|| for `stag` iterations: the float32 CG has
    // reached its accuracy; the float64 Newton residual takes over
    st->rr = rr_new;
    st->done = 1;
  } else if (st->it >= st->maxit) {
    st->rr = rr_new;
    st->status = RVE_DEV_ERR_CG_MAXIT;
    st->done = 1;
  } else {
    st->beta = rr_new / st->rr;
    st->rr = rr_new;
  }
  if (rr_new < 0.81 * st->rr_min) {
    st->rr_min = rr_new;
    st->it_min = st->it;
  }
}

// CG start once b.b of the right-hand side b = r (x = 0) is known (one
// thread): stopping threshold max(tol^2 b.b, atol^2), counters reset.
RVE_DEV void cg_after_bb(SolverState* st, double bb) {
  st->bb = bb;
  st->rr = bb;
  st->rr_min = bb;
  st->it_min = 0;
  st->it = 0;
  st->beta = 0.0;
  st->status = 0;
  st->tol2 = fmax(st->cg_tol * st->cg_tol * bb, st->cg_atol * st->cg_atol);
  st->done = (bb == 0.0) ? 1 : 0;
  if (!isfinite(bb)) {
    st->status = RVE_DEV_ERR_NONFINITE;
    st->done = 1;
  }
}

// ---------------------------------------------------------------------------
// Deterministic block reduction of NV doubles: warp xor-butterflies in a fixed
// pattern, then one fixed tree over the warps.  Result valid in all threads.
// ---------------------------------------------------------------------------
template <int NV>
RVE_DEV void block_sum(double (&v)[NV]) {
  __shared__ double red[32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[warp][k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w][k];  // same order in every thread
    v[k] = s;
  }
  __syncthreads();
}

// Writes this block's NV partial sums to partials[block*NV + k]; the block
// that finishes last sums all partials in a fixed order (deterministic,
// independent of which block is last) into total[k] and returns true.
// The reduction over `nblk` thread blocks that call it with their index
// `bid` (a batched launch runs several such groups, one per cell).
template <int NV>
RVE_DEV bool last_block_sum_of(double (&v)[NV], double* partials, unsigned int* counter,
                               double (&total)[NV], unsigned int bid, unsigned int nblk) {
  __shared__ bool am_last;
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[(size_t)bid * NV + k] = v[k];
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    am_last = (prev == nblk - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double s[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) s[k] = 0.0;
  for (unsigned int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NV; ++k) s[k] += __ldcg(partials + (size_t)b * NV + k);
  block_sum<NV>(s);
#pragma unroll
  for (int k = 0; k < NV; ++k) total[k] = s[k];
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

template <int NV>
RVE_DEV bool last_block_sum(double (&v)[NV], double* partials, unsigned int* counter,
                            double (&total)[NV]) {
  return last_block_sum_of<NV>(v, partials, counter, total,
                               blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z),
                               gridDim.x * gridDim.y * gridDim.z);
}

// ---------------------------------------------------------------------------
// Material views.  Either a phase index per voxel with a per-phase table, or
// per-voxel parameter arrays.  SVK parameters: lambda, mu.
// ---------------------------------------------------------------------------
template <typename R>
struct MatView {
  const uint8_t* phase;  // [n] or null
  const R* table;        // [nphase][nparam] when phase != null
  const R* vox;          // [nparam][n] when phase == null
  int nparam;
  size_t n;
  RVE_DEV R get(size_t v, int k) const {
    if (phase) return table[(int)phase[v] * nparam + k];
    return vox[(size_t)k * n + v];
  }
};
