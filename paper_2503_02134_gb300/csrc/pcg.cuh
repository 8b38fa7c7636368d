// Launchers of the PCG vector kernels (pcg_kernels.cu).
#pragma once

#include "reduce.cuh"

namespace sem {

int vec_grid(const Handle& h, int64_t L);
int launch_cg_update64(Handle& h, double* x, double* r, const double* p, const double* w,
                       PcgScalars* s, double* hist);
int launch_cg_update32(Handle& h, int dm, float* x, float* r, const float* p, const float* w,
                       const float* minv, PcgScalars* s, double* hist);
int launch_cg_init64(Handle& h, double* r, const double* b, const double* ax, const double* minv,
                     PcgScalars* s, double* hist);
int launch_cg_init32(Handle& h, int dm, float* r, const float* b, const float* ax,
                     const float* minv, PcgScalars* s, double* hist);
int launch_cast64to32(Handle& h, const double* a, float* b);
int launch_cast32to64(Handle& h, const float* a, double* b);
int launch_add32to64(Handle& h, double* x, const float* d);
int launch_masked_copy64(Handle& h, const double* src, double* dst);
int launch_masked_copy32(Handle& h, const double* src, float* dst);
int launch_cg_replace32(Handle& h, int dm, const double* r64, float* r32, const float* minv,
                        double tol, PcgScalars* s);
int launch_set_bnorm(Handle& h, PcgScalars* s, double bnorm, double* hist);
int launch_scal_setup(Handle& h, PcgScalars* s, double tol, int maxit, int fixed, int stag_window);

}  // namespace sem
