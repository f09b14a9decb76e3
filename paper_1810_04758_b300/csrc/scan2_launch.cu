// scan2_launch.cu -- the instances of the neighbour-cell scan kernel k_scan2
// for one dimension, KNN_SCAN2_DIM (set by the build: one object per d), and
// their launcher (interface in scan2_launch.h).
#include <algorithm>
#include <mutex>
#include <vector>

#include "scan2.cuh"
#include "scan2_launch.h"

#ifndef KNN_SCAN2_DIM
#error "build this unit with -DKNN_SCAN2_DIM=d (1 <= d <= 8)"
#endif

// Everything below but the specialisations of the interface lives in a
// namespace of its own per unit: the units share one source file, so names
// in an anonymous namespace, and template instances such as launch_one<E,
// MEGA>, would otherwise collide (or be merged) across units at link time.
#define KNN_S2_CAT2(a, b) a##b
#define KNN_S2_CAT(a, b) KNN_S2_CAT2(a, b)
#define KNN_S2_NS KNN_S2_CAT(scan2_unit_d, KNN_SCAN2_DIM)

namespace knn {
namespace KNN_S2_NS {

constexpr int DIM = KNN_SCAN2_DIM;

// Fill the nearest-first neighbour order g_nb_order (this unit's copy) on
// the current device: for each d the base-3 offset codes ordered by how many
// dimensions move.
cudaError_t ensure_nb_order(int dev)
{
    static std::mutex mu;
    static bool done[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev & 63]) return cudaSuccess;
    std::vector<uint16_t> tab;
    tab.reserve(NB_ORDER_TOTAL);
    for (int d = 1; d <= MAX_DIM; ++d) {
        int no = 1;
        for (int k = 0; k < d; ++k) no *= 3;
        std::vector<std::pair<int, int>> v;
        for (int o = 0; o < no; ++o) {
            int moves = 0, r = o;
            for (int k = 0; k < d; ++k) {
                moves += (r % 3) != 1;
                r /= 3;
            }
            v.push_back({moves, o});
        }
        std::stable_sort(v.begin(), v.end());
        for (auto &e : v) tab.push_back((uint16_t)e.second);
    }
    cudaError_t e = cudaMemcpyToSymbol(g_nb_order, tab.data(), tab.size() * sizeof(uint16_t));
    if (e == cudaSuccess) done[dev & 63] = true;
    return e;
}

template <int E, bool MEGA>
cudaError_t launch_one(const ScanArgs &a, size_t smem, cudaStream_t s, int nsm, int dev, bool *nofit,
                       int64_t *launches)
{
    constexpr int QM = scan2_queries_per_item(E);
    static bool configured[64] = {};
    cudaError_t e = ensure_nb_order(dev);
    if (e != cudaSuccess) return e;
    if (!configured[dev & 63]) {
        e = cudaFuncSetAttribute(k_scan2<DIM, QM, E, MEGA>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        configured[dev & 63] = true;
    }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_scan2<DIM, QM, E, MEGA>, S2_CTA, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) {
        *nofit = true;
        return cudaSuccess;
    }
    const unsigned grid = (unsigned)std::min<int64_t>(((int64_t)a.nitems + S2_WARPS - 1) / S2_WARPS,
                                                      (int64_t)occ * nsm);
    if (grid == 0) return cudaSuccess;
    k_scan2<DIM, QM, E, MEGA><<<grid, S2_CTA, smem, s>>>(a);
    ++*launches;
    return cudaGetLastError();
}

template <int E, bool MEGA>
cudaError_t launch_multi(const MultiScanArgs &p, size_t smem, cudaStream_t s, int nsm, int dev, bool *nofit,
                         int64_t *launches)
{
    constexpr int QM = scan2_queries_per_item(E);
    static bool configured[64] = {};
    cudaError_t e = ensure_nb_order(dev);
    if (e != cudaSuccess) return e;
    if (!configured[dev & 63]) {
        e = cudaFuncSetAttribute(k_scan2_multi<DIM, QM, E, MEGA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024);
        if (e != cudaSuccess) return e;
        configured[dev & 63] = true;
    }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_scan2_multi<DIM, QM, E, MEGA>, S2_CTA, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) {
        *nofit = true;
        return cudaSuccess;
    }
    const unsigned grid = (unsigned)std::min<int64_t>(((int64_t)p.nuitems + S2_WARPS - 1) / S2_WARPS,
                                                      (int64_t)occ * nsm);
    if (grid == 0) return cudaSuccess;
    k_scan2_multi<DIM, QM, E, MEGA><<<grid, S2_CTA, smem, s>>>(p);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace KNN_S2_NS

using KNN_S2_NS::DIM;
using KNN_S2_NS::launch_multi;
using KNN_S2_NS::launch_one;

template <>
cudaError_t scan2_launch<DIM>(const ScanArgs &a, int E, bool mega, size_t smem, cudaStream_t s, int nsm, int dev,
                              bool *nofit, int64_t *launches)
{
    *nofit = false;
    switch (E * 2 + (mega ? 1 : 0)) {
    case 4: return launch_one<2, false>(a, smem, s, nsm, dev, nofit, launches);
    case 5: return launch_one<2, true>(a, smem, s, nsm, dev, nofit, launches);
    case 8: return launch_one<4, false>(a, smem, s, nsm, dev, nofit, launches);
    case 9: return launch_one<4, true>(a, smem, s, nsm, dev, nofit, launches);
    case 16: return launch_one<8, false>(a, smem, s, nsm, dev, nofit, launches);
    case 17: return launch_one<8, true>(a, smem, s, nsm, dev, nofit, launches);
    default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t scan2_launch_multi<DIM>(const MultiScanArgs &p, int E, bool mega, size_t smem, cudaStream_t s, int nsm,
                                    int dev, bool *nofit, int64_t *launches)
{
    *nofit = false;
    switch (E * 2 + (mega ? 1 : 0)) {
    case 4: return launch_multi<2, false>(p, smem, s, nsm, dev, nofit, launches);
    case 5: return launch_multi<2, true>(p, smem, s, nsm, dev, nofit, launches);
    case 8: return launch_multi<4, false>(p, smem, s, nsm, dev, nofit, launches);
    case 9: return launch_multi<4, true>(p, smem, s, nsm, dev, nofit, launches);
    case 16: return launch_multi<8, false>(p, smem, s, nsm, dev, nofit, launches);
    case 17: return launch_multi<8, true>(p, smem, s, nsm, dev, nofit, launches);
    default: return cudaErrorInvalidValue;
    }
}

template <>
unsigned scan2_check_word<DIM>(bool clear)
{
#ifdef KNN_CHECKS
    unsigned w = 0, z = 0;
    if (cudaMemcpyFromSymbol(&w, g_check_word, sizeof(w)) != cudaSuccess) return 0xffffffffu;
    if (clear && w) cudaMemcpyToSymbol(g_check_word, &z, sizeof(z));
    return w;
#else
    (void)clear;
    return 0;
#endif
}

template <>
cudaError_t scan2_debug_read<DIM>(unsigned long long *out, bool reset)
{
#ifdef KNN_PHASE_TIMING
    unsigned long long ph[16], cn[16];
    cudaError_t e = cudaMemcpyFromSymbol(ph, g_phase, sizeof(ph));
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(cn, g_count, sizeof(cn));
    if (e != cudaSuccess) return e;
    for (int i = 0; i < 16; ++i) {
        // per-item maxima combine by max, everything else by sum
        out[i] = (i == 8 || i == 11 || i == 13) ? std::max(out[i], ph[i]) : out[i] + ph[i];
        out[16 + i] += cn[i];
    }
    if (reset) {
        unsigned long long z[16] = {};
        e = cudaMemcpyToSymbol(g_phase, z, sizeof(z));
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_count, z, sizeof(z));
    }
    return e;
#else
    (void)out;
    (void)reset;
    return cudaSuccess;
#endif
}

}  // namespace knn
