// Drivers built on the Arnoldi kernels: restarted GMRES / iterative refinement and
// Krylov-Schur.
#include "kc_internal.cuh"

extern "C" {

kc_status gmres_solve(kc_ctx* ctx, const kc_csr* A, const kc_csr* A32, const double* b,
                      double* x, const kc_gmres_opts* opts, kc_gmres_info* info) {
  (void)A; (void)A32; (void)b; (void)x; (void)opts; (void)info;
  return kc::fail(ctx, KC_ERR_INVALID_ARG, "gmres_solve: not available in this build");
}

kc_status krylov_schur_eigs(kc_ctx* ctx, const kc_csr* A, const double* v0,
                            const kc_ks_opts* opts, double* eig_re, double* eig_im,
                            double* resid, int* nconv, int* restarts, int* matvecs) {
  (void)A; (void)v0; (void)opts; (void)eig_re; (void)eig_im; (void)resid; (void)nconv;
  (void)restarts; (void)matvecs;
  return kc::fail(ctx, KC_ERR_INVALID_ARG, "krylov_schur_eigs: not available in this build");
}

}  // extern "C"
