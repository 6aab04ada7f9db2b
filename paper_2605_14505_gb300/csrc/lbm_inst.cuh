// Instantiation helper: defines the kernel table of one (pair, storage).
#pragma once

#include "lbm_dispatch.h"
#include "lbm_kernels.cuh"
#include "lbm_stage.cuh"

#define LBM_STEP_PAIR(P, F, T) {(const void*)k_step<P, F, T, false>, (const void*)k_step<P, F, T, true>}
#define LBM_STEP2_PAIR(P, F, T) {lbm::step2_ptr<P, F, T, false>(), lbm::step2_ptr<P, F, T, true>()}
#define LBM_STAGED_PAIR(P, F, T) {lbm::staged_ptr<P, F, T, false>(), lbm::staged_ptr<P, F, T, true>()}
#define LBM_STEPD_PAIR(P, F, T) {(const void*)k_step_diag<P, F, T, false>, (const void*)k_step_diag<P, F, T, true>}
#define LBM_STEP2D_PAIR(P, F, T) {lbm::step2d_ptr<P, F, T, false>(), lbm::step2d_ptr<P, F, T, true>()}

namespace lbm {
// Two-nodes-per-thread kernel for 16-bit storage; FP32 tables hold null (and
// never instantiate it).
template <class P, int F, class T, bool ODD>
inline const void* step2_ptr()
{
    if constexpr (std::is_same<T, float>::value)
        return nullptr;
    else
        return (const void*)k_step2<P, F, T, ODD>;
}
template <class P, int F, class T, bool ODD>
inline const void* step2d_ptr()
{
    if constexpr (std::is_same<T, float>::value)
        return nullptr;
    else
        return (const void*)k_step2_diag<P, F, T, ODD>;
}
template <class P, int F, class T, bool ODD>
inline const void* staged_ptr()
{
    if constexpr (std::is_same<T, float>::value)
        return nullptr;
    else
        return (const void*)k_step_staged<P, F, T, ODD>;
}
}  // namespace lbm

#define LBM_DEFINE_KERNEL_SET(NAME, QF_, QG_, T)                                                   \
    namespace lbm {                                                                               \
    const KernelSet* NAME()                                                                       \
    {                                                                                             \
        using P = Pair<QF_, QG_>;                                                                 \
        static const KernelSet ks = {                                                             \
            QF_,                                                                                  \
            QG_,                                                                                  \
            {LBM_STEP_PAIR(P, 0, T), LBM_STEP_PAIR(P, 1, T), LBM_STEP_PAIR(P, 2, T),              \
             LBM_STEP_PAIR(P, 3, T)},                                                             \
            {LBM_STEP2_PAIR(P, 0, T), LBM_STEP2_PAIR(P, 1, T), LBM_STEP2_PAIR(P, 2, T),           \
             LBM_STEP2_PAIR(P, 3, T)},                                                            \
            {LBM_STAGED_PAIR(P, 0, T), LBM_STAGED_PAIR(P, 1, T), LBM_STAGED_PAIR(P, 2, T),        \
             LBM_STAGED_PAIR(P, 3, T)},                                                           \
            {LBM_STEPD_PAIR(P, 0, T), LBM_STEPD_PAIR(P, 1, T), LBM_STEPD_PAIR(P, 2, T),           \
             LBM_STEPD_PAIR(P, 3, T)},                                                            \
            {LBM_STEP2D_PAIR(P, 0, T), LBM_STEP2D_PAIR(P, 1, T), LBM_STEP2D_PAIR(P, 2, T),        \
             LBM_STEP2D_PAIR(P, 3, T)},                                                           \
            (const void*)k_init_fields<P, T>,                                                     \
            (const void*)k_init_tgv<P, T>,                                                        \
            (const void*)k_get_pops<P, T>,                                                        \
            (const void*)k_set_pops<P, T>,                                                        \
            (const void*)k_diag_moments<P, T>,                                                    \
            (const void*)k_get_fields<P, T>,                                                      \
            (const void*)k_sample_pops<P, T>,                                                     \
        };                                                                                        \
        return &ks;                                                                               \
    }                                                                                             \
    }
