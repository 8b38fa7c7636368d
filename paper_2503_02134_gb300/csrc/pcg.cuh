// Launchers of the PCG vector kernels (pcg_kernels.cu).
#pragma once

#include "reduce.cuh"

namespace sem {

// Scalars update after the reductions of an iteration (one thread).
__device__ inline void finish_iteration(PcgScalars* s, double rtr, double rtz_new, double* hist) {
  s->iter += 1;
  s->rtr = rtr;
  const double relres = sqrt(rtr) / s->bnorm;
  s->relres = relres;
  if (hist) hist[s->iter] = relres;
  if (!isfinite(relres)) {
    s->status = SEM_BREAKDOWN;
    s->done = 1;
  } else if (s->fixed) {
    if (s->iter >= s->maxit) s->done = 1;
  } else if (relres <= s->tol) {
    s->done = 1;
  } else if (s->iter >= s->maxit) {
    s->status = SEM_MAXIT;
    s->done = 1;
  } else if (s->stag_window > 0) {
    if (rtr < 0.81 * s->best_rtr) {   // ||r|| fell by 10 %
      s->best_rtr = rtr;
      s->best_it = s->iter;
    } else if (s->iter - s->best_it >= s->stag_window) {
      s->status = SEM_STAGNATED;
      s->done = 1;
    }
  }
  s->beta = rtz_new / s->rtz;
  s->rtz_old = s->rtz;
  s->rtz = rtz_new;
}


int vec_grid(const Handle& h, int64_t L);
int launch_cg_update64(Handle& h, double* x, double* r, const double* p, const double* w,
                       PcgScalars* s, double* hist);
int launch_cg_update32(Handle& h, int dm, float* x, float* r, const float* p, const float* w,
                       const float* minv, PcgScalars* s, double* hist);
bool gs_fusable(const Handle& h);
int launch_cg_update32_gs(Handle& h, int dm, int acc, float* x, float* r, const float* p,
                          const float* w, const float* minv, PcgScalars* s, double* hist);
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
