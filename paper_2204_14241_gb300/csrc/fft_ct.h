// FP32 FFT passes with compile-time lengths (fft_ct.cu).
#pragma once

#include "internal.h"

namespace hmc {

constexpr int kFftcXUpd = 1;   // x-axis pass fused with the CG update (forward)
constexpr int kFftcXDot = 2;   // x-axis inverse pass fused with the <r, z> dot

bool fftc_supported(int n);
// true if an axis pass of length n over an inner extent `inner` has a compiled kernel
bool fftc_can(int n, int64_t inner);
int fftc_axis(hmc_ctx* ctx, float2* data, int64_t outer, int n, int64_t inner, int dir, const float2* src,
              const CgScalars* cgs, int64_t opr);
int fftc_precond_tau(hmc_ctx* ctx, const Lat& lat, float2* y, int nrhs, const CgScalars* cgs, const PcTables* pt);
int fftc_x_cg(hmc_ctx* ctx, const Lat& lat, int mode, const float2* src, float2* dst, float2* x, float2* r,
              const float2* p, const float2* q, int nrhs, const CgScalars* cgs, double* part, int* nblk_out);

}  // namespace hmc
