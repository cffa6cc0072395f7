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
// cosk: the cos k table indexed by the position of k along x and y (pt->cosk32 for natural
// order, pt->cosk32_xy after the (x, y) pass of fftc_xy_cg)
// part (optional): partial sums of sum P-hat |y-hat|^2 = <y_in, P y_in> when the transform
// ahead of this pass is unitary; *nblk_out of them per right-hand side. band_major: y is the
// spectrum the forward (x, y) pass leaves, [nrhs][Nt][band][L * L][spin], not the site layout
// [nrhs][Nt][L * L][band][spin].
int fftc_precond_tau(hmc_ctx* ctx, const Lat& lat, float2* y, int nrhs, const CgScalars* cgs, const PcTables* pt,
                     const float* cosk, double* part, int* nblk_out, bool band_major);
int fftc_x_cg(hmc_ctx* ctx, const Lat& lat, int mode, const float2* src, float2* dst, float2* x, float2* r,
              const float2* p, const float2* q, int nrhs, const CgScalars* cgs, double* part, int* nblk_out);

// in-place tau pass for these lengths (spectrum in digit-permuted order inside the kernel)
bool fftc_tau_supported(int n);
// frequency index held at position pos after the forward steps of that pass
int fftc_tau_freq(int n, int pos);
// (x, y) passes in one kernel per band and plane, for lattice extents with a compiled split
bool fftc_xy_supported(int L);
// frequency index held at position pos of an axis after the forward (x, y) pass
int fftc_xy_freq(int L, int pos);
// dst = F_xy src (dir < 0, permuted order out) or F_xy^-1 src (dir > 0, permuted order in);
// right-hand sides with cgs[k].active == 0 are skipped when cgs is given. The spectrum (dst of
// the forward pass, src of the inverse) is band-major: [nrhs][Nt][band][L * L][spin], so that
// each block's band of a plane is one contiguous 16 L^2-byte run; src and dst must not overlap
// (HMC_ERR_ARG).
int fftc_xy_apply(hmc_ctx* ctx, const Lat& lat, const float2* src, float2* dst, int nrhs, int dir,
                  const CgScalars* cgs);
// pnew = F_xy^-1 zhat + beta_k pold for every active right-hand side (beta from cgs); zhat
// band-major as above
int fftc_xy_inverse_pupd(hmc_ctx* ctx, const Lat& lat, const float2* zhat, const float2* pold, float2* pnew, int nrhs,
                         const CgScalars* cgs);
// x += alpha p, r -= alpha q with partial ||r||^2 (*nblk_out = 2 Nt per right-hand side)
int fftc_xy_update(hmc_ctx* ctx, const Lat& lat, float2* x, float2* r, const float2* p, const float2* q, int nrhs,
                   const CgScalars* cgs, double* part, int* nblk_out);

}  // namespace hmc
