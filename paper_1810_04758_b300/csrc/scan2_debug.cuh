// scan2_debug.cuh -- diagnostic phase timing and event counts of k_scan2.
//
// Built with -DKNN_PHASE_TIMING, lane 0 of every warp adds clock64() deltas
// per phase of the scan kernel to g_phase and per-warp event counts to
// g_count (read back and cleared by knnjoin_debug_phases); otherwise every
// marker compiles to nothing and the kernel is unchanged.  The state lives in
// a DebugState that the kernel declares (KNN_PT_DECL) and hands to the
// functions it calls (KNN_CNT_PARAM / KNN_CNT_ARG).
#pragma once

#ifdef KNN_PHASE_TIMING
namespace knn {
// g_phase: [0, 8) cycles per phase; per item: [8] max cycles, [9] sum,
// [10] count, [11] max query-tiles, [12] sum of Q, [13] max cycles / [14]
// sum / [15] count of items with Q <= 2.
__device__ unsigned long long g_phase[16];
// g_count: event counts (meaning set by the KNN_CNT sites of the kernel).
__device__ unsigned long long g_count[16];
struct DebugState {
    unsigned long long ph[8], pt, cn[16];
};
}  // namespace knn
#define KNN_PT_DECL                          \
    ::knn::DebugState dbg_;                  \
    for (int q_ = 0; q_ < 8; ++q_) dbg_.ph[q_] = 0; \
    for (int q_ = 0; q_ < 16; ++q_) dbg_.cn[q_] = 0; \
    dbg_.pt = clock64()
#define KNN_PT(i)                          \
    do {                                   \
        unsigned long long t_ = clock64(); \
        dbg_.ph[i] += t_ - dbg_.pt;        \
        dbg_.pt = t_;                      \
    } while (0)
#define KNN_CNT(i, v)                            \
    do {                                         \
        dbg_.cn[i] += (unsigned long long)(v);   \
    } while (0)
// cycles of a stretch of code added to event count i
#define KNN_CYC_BEGIN(nm) const unsigned long long nm##_c0 = clock64()
#define KNN_CYC_END(nm, i) KNN_CNT(i, clock64() - nm##_c0)
// extra parameter / argument that hands the state to called functions
#define KNN_CNT_PARAM , ::knn::DebugState &dbg_
#define KNN_CNT_ARG , dbg_
#define KNN_PT_FLUSH                                                          \
    do {                                                                      \
        if ((threadIdx.x & 31) == 0) {                                        \
            for (int q_ = 0; q_ < 8; ++q_) atomicAdd(&g_phase[q_], dbg_.ph[q_]); \
            for (int q_ = 0; q_ < 16; ++q_)                                   \
                if (dbg_.cn[q_]) atomicAdd(&g_count[q_], dbg_.cn[q_]);        \
        }                                                                     \
    } while (0)
#define KNN_ITEM_BEGIN unsigned long long it0_ = clock64(), itq_ = 0
#define KNN_ITEM_TILE(x) itq_ += (x)
#define KNN_ITEM_END(Q)                                      \
    do {                                                     \
        if ((threadIdx.x & 31) == 0) {                       \
            const unsigned long long dt_ = clock64() - it0_; \
            atomicMax(&g_phase[8], dt_);                     \
            atomicAdd(&g_phase[9], dt_);                     \
            atomicAdd(&g_phase[10], 1ull);                   \
            atomicMax(&g_phase[11], itq_);                   \
            atomicAdd(&g_phase[12], (unsigned long long)(Q)); \
            if ((Q) <= 2) {                                  \
                atomicMax(&g_phase[13], dt_);                \
                atomicAdd(&g_phase[14], dt_);                \
                atomicAdd(&g_phase[15], 1ull);               \
            }                                                \
        }                                                    \
    } while (0)
#else
#define KNN_PT_DECL
#define KNN_PT(i) \
    do {          \
    } while (0)
#define KNN_CNT(i, v) \
    do {              \
    } while (0)
#define KNN_CYC_BEGIN(nm)
#define KNN_CYC_END(nm, i) \
    do {                   \
    } while (0)
#define KNN_CNT_PARAM
#define KNN_CNT_ARG
#define KNN_PT_FLUSH \
    do {             \
    } while (0)
#define KNN_ITEM_BEGIN
#define KNN_ITEM_TILE(x) \
    do {                 \
    } while (0)
#define KNN_ITEM_END(Q) \
    do {                \
    } while (0)
#endif
