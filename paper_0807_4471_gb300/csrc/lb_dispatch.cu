// lb_dispatch.cu -- precision dispatch of the kernel launchers and the
// launch geometry queries used by the host code.
#include "lb_internal.h"
#include "lb_layout.cuh"

namespace lbgb {

#define LB_SWITCH(P_, EXPR)                       \
    switch (P_) {                                 \
        case LB_FP64: { constexpr int P = LB_FP64; EXPR; } \
        case LB_FP32: { constexpr int P = LB_FP32; EXPR; } \
        case LB_FP16_OFFSET: { constexpr int P = LB_FP16_OFFSET; EXPR; } \
        case LB_BF16_OFFSET: { constexpr int P = LB_BF16_OFFSET; EXPR; } \
    }

int kernel_smem_bytes(int p) { LB_SWITCH(p, return Layout<P>::SMEM) return 0; }
int kernel_tile_x(int p) { LB_SWITCH(p, return Layout<P>::TX) return 0; }
int kernel_tile_y(int p) { LB_SWITCH(p, return Layout<P>::TY) return 0; }
int kernel_ghost_x(int p) { LB_SWITCH(p, return Layout<P>::GX) return 0; }
int kernel_elem_bytes(int p) { LB_SWITCH(p, return (int)sizeof(typename Layout<P>::T)) return 0; }
int kernel_smem_obs_bytes(int p) { LB_SWITCH(p, return Layout<P>::SMEM_OBS) return 0; }
int kernel_block_rows(int p) { LB_SWITCH(p, return Layout<P>::TYB) return 0; }
int kernel_scale_log2(int p) { LB_SWITCH(p, return Prec<P>::SCALE_LOG2) return 0; }
template <int P>
static int staged_of(int spt) {
    if constexpr (Prec<P>::NB2 > 0)
        if (spt == 2) return Layout<P, 2>::STAGED ? 1 : 0;
    return Layout<P, 1>::STAGED ? 1 : 0;
}
int kernel_staged(int p, int spt) { LB_SWITCH(p, return staged_of<P>(spt)) return 1; }

cudaError_t launch_step(int precision, const void* args, int variant, int spt, dim3 grid,
                        cudaStream_t s) {
    LB_SWITCH(precision, return launch_step_prec<P>(args, variant, spt, grid, s))
    return cudaErrorInvalidValue;
}

cudaError_t kernels_configure(int precision) {
    LB_SWITCH(precision, return configure_prec<P>())
    return cudaErrorInvalidValue;
}

cudaError_t launch_observe(int precision, const CUtensorMap* tin, const void* args, dim3 grid,
                           cudaStream_t s) {
    LB_SWITCH(precision, return launch_observe_prec<P>(tin, args, grid, s))
    return cudaErrorInvalidValue;
}

cudaError_t launch_init_seeded(int precision, const Geom& g, const void* coef, void* fout,
                               double rho0, double amp, double u_wall, int init_shear,
                               unsigned long long seed, cudaStream_t s) {
    LB_SWITCH(precision, return launch_init_prec<P>(g, coef, fout, 0, nullptr, rho0, amp, u_wall,
                                                    init_shear, seed, s))
    return cudaErrorInvalidValue;
}

cudaError_t launch_init_fields(int precision, const Geom& g, const void* coef, void* fout,
                               const double* fields, cudaStream_t s) {
    LB_SWITCH(precision, return launch_init_prec<P>(g, coef, fout, 1, fields, 0, 0, 0, 0, 0, s))
    return cudaErrorInvalidValue;
}

cudaError_t launch_load_pops(int precision, const Geom& g, const void* coef, void* fout,
                             const double* pops, int i0, int i1, cudaStream_t s) {
    LB_SWITCH(precision, return launch_load_pops_prec<P>(g, coef, fout, pops, i0, i1, s))
    return cudaErrorInvalidValue;
}

#undef LB_SWITCH

}  // namespace lbgb
