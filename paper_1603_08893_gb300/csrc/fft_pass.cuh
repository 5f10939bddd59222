// Pieces shared by the FFT pass kernels (kernels_fft.cu, kernels_fft4.cu).
#pragma once
#include "kernels.h"

#define FFT_THREADS 256
// float kernels: three CTAs per SM (<= 85 registers); double: two (<= 128)
#define FFT_BOUNDS(R) __launch_bounds__(FFT_THREADS, sizeof(R) == 4 ? 3 : 2)

template <typename R>
RVE_DEV R signed_freq(int k, int n) {
  return (R)((k <= (n - 1) / 2) ? k : k - n);
}

template <typename R>
struct LineParams {
  GridGeom g;
  int t, grp;  // kz tile and groups (y pass)
  double scale;
  cplx<R>* spec;
  const int* done;
  const cplx<R>* tw;
};

// ---------------------------------------------------------------------------
// 16-byte asynchronous global->shared copies (cp.async): a tile's loads are
// in flight while the previous tile is transformed.  bytes = 0 zero-fills.
// ---------------------------------------------------------------------------
RVE_DEV void cp_async16(void* sdst, const void* gsrc, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(bytes));
}
RVE_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
RVE_DEV void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Tiles of the strided passes: `rows` rows of T complex values (T a power of
// two, 64 bytes); row r of the tile starts at gbase + r * rstride.  Rows are
// copied in 16-byte chunks; chunks past the padded row length are zero-filled
// and not read.
template <typename R>
RVE_DEV void issue_tile(cplx<R>* sbuf, const cplx<R>* gbase, size_t rstride, int rows, int T,
                        int ts, int kz0, int hzp, const cplx<R>* any_valid) {
  constexpr int EPC = 16 / sizeof(cplx<R>);  // complex values per chunk
  const int cpr = T / EPC;                   // chunks per row (power of two)
  const int cs = __ffs(cpr) - 1;
  const int nch = rows * cpr;
  for (int c = threadIdx.x; c < nch; c += blockDim.x) {
    const int row = c >> cs;
    const int t = (c & (cpr - 1)) * EPC;
    const bool ok = (kz0 + t) < hzp;
    const cplx<R>* src = ok ? gbase + (size_t)row * rstride + t : any_valid;
    cp_async16(sbuf + (row << ts) + t, src, ok ? 16 : 0);
  }
}

