// vector_kernels.h -- declarations of the setup and vector kernels (vector_kernels.cu).
#pragma once

#include "internal.h"

namespace feod {

constexpr int RED_BLOCKS = 1216;    // fixed reduction grid (8 x 152): results do not depend on the GPU
constexpr int RED_THREADS = 256;
constexpr int VEC_BLOCKS = 1216;
constexpr int VEC_THREADS = 256;

enum CgDone : int { CG_RUNNING = 0, CG_CONVERGED = 1, CG_BREAKDOWN = 2, CG_NAN = 3, CG_MAXIT = 4 };

// Device-resident CG scalars.  `done` != 0 makes every later kernel of a queued batch a no-op.
struct CgState {
    double rz, rr, rr0, tol2, pq, alpha, beta;
    int iter, max_iter;
    int done;
    unsigned counter;      // last-block ticket of the reductions (returns to 0 after each)
    int scale_exp;         // FP32 CG: the system is solved for b / 2^scale_exp
    double scalar;         // result slot of plain dot products
    int xpend;             // FP64-vector CG: the x update of the last iteration is still due
};

// One face of a context's DOF lattice (see k_face_add).
struct FaceParams {
    int dim, face, natural;
    int64_t m[3];
};

__global__ void k_axpby(double alpha, const double *__restrict__ x, double beta, double *__restrict__ y, int64_t n);
__global__ void k_mul(const double *__restrict__ d, const double *__restrict__ r, double *__restrict__ z, int64_t n);
__global__ void k_recip(const double *__restrict__ x, double *__restrict__ y, int64_t n);
__global__ void k_face_add(FaceParams F, double *__restrict__ y, const double *__restrict__ buf);
__global__ void k_geometry(const GeomParams G, const double *__restrict__ vert, double *__restrict__ geo,
                           int *__restrict__ err);
__global__ void k_node_coords(const GeomParams G, int k, const double *__restrict__ vert, double *__restrict__ xyz,
                              int64_t nl);
__global__ void k_design_factors(const GeomParams G, const double *__restrict__ rho, double kappa_eps,
                                 double kappa_q, double *__restrict__ kr, double *__restrict__ dkr);
__global__ void k_dot(const double *__restrict__ a, const double *__restrict__ b, int64_t n, double *partial,
                      unsigned *counter, double *out);
__global__ void k_cg_init(const double *__restrict__ b, const double *__restrict__ dinv, double *__restrict__ x,
                          double *__restrict__ r, double *__restrict__ p, float *__restrict__ p32, int64_t n,
                          CgState *st, double rtol, int max_iter, double *partial);
__global__ void k_cg_alpha(const double *__restrict__ p, const double *__restrict__ q, int64_t n, CgState *st,
                           double *partial);
__global__ void k_cg_update(double *__restrict__ r, const double *__restrict__ q, const double *__restrict__ dinv,
                            double *__restrict__ z, int64_t n, CgState *st, double *partial);
__global__ void k_cg_direction(double *__restrict__ x, double *__restrict__ p, float *__restrict__ p32,
                               const double *__restrict__ z, const double *__restrict__ r, int64_t n,
                               CgState *st, double *partial);
__global__ void k_waxpy(double *__restrict__ y, const double *__restrict__ a, double alpha,
                        const double *__restrict__ b, int64_t n);
__global__ void k_scale(double *__restrict__ y, const double *__restrict__ x, double alpha, int64_t n);
__global__ void k_reciprocal(float *__restrict__ y, double *__restrict__ y64, const double *__restrict__ x, int64_t n);
__global__ void k_split_df(const double *__restrict__ x, dfloat *__restrict__ y, int64_t n);
__global__ void k_cg_init32(const double *__restrict__ b, const float *__restrict__ dinv, float *__restrict__ x,
                            float *__restrict__ r, float *__restrict__ p, int64_t n, CgState *st, const double *bb,
                            double rtol, int max_iter, double *partial);
__global__ void k_cg_alpha32(const float *__restrict__ p, const float *__restrict__ q, int64_t n, CgState *st,
                             double *partial);
__global__ void k_cg_update32(float *__restrict__ x, float *__restrict__ r, const float *__restrict__ p,
                              const float *__restrict__ q, const float *__restrict__ dinv, int64_t n, CgState *st,
                              double *partial);
__global__ void k_cg_direction32(float *__restrict__ p, const float *__restrict__ r, const float *__restrict__ dinv,
                                 int64_t n, const CgState *st);
__global__ void k_wait_selftest(int *err);
__global__ void k_cg_continue(cudaGraphConditionalHandle h, const CgState *st);
__global__ void k_scale_rhs(double *__restrict__ y, const double *__restrict__ b, int64_t n, const double *bb,
                            CgState *st);
__global__ void k_unscale(double *__restrict__ x, int64_t n, const CgState *st);
__global__ void k_cg_widen(double *__restrict__ y, const float *__restrict__ x, int64_t n, const CgState *st);

}  // namespace feod
