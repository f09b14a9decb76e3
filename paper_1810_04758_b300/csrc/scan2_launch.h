// scan2_launch.h -- host interface of the neighbour-cell scan kernel k_scan2
// (scan2.cuh).  The kernel's instances for each dimension d are compiled in
// their own translation unit (scan2_launch.cu built with KNN_SCAN2_DIM = d),
// so the library builds in parallel; each unit holds its own copies of the
// kernel's device tables and reports through the functions declared here.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace knn {

struct ScanArgs;
struct MultiScanArgs;

// Warps per CTA of k_scan2 (each works alone on its own work items).
constexpr int S2_WARPS = 4;
constexpr int S2_CTA = S2_WARPS * 32;

// Row of a query in shared memory: coordinates, current threshold, sorted
// position (as float bits), padded to a multiple of 4 floats (vector loads).
__host__ __device__ constexpr int query_row_floats(int d) { return (d + 2 + 3) & ~3; }

// Smallest d whose tiles score the item's queries two at a time (packed
// FP32: one 64-bit register holds a coordinate of queries 2p and 2p + 1),
// with buffers of at most 32 * S2_QPAIR_MAXE entries.  Measured on 2M-point
// sets: 4% faster at d = 6 with the 64-entry buffers of K <= 32 (16 queries
// per item), 7-8% slower at d = 4 and 7-12% slower with the 8-query items of
// larger buffers, slower at d = 2.
#ifndef S2_QPAIR_DIM
#define S2_QPAIR_DIM 6
#endif
#ifndef S2_QPAIR_MAXE
#define S2_QPAIR_MAXE 2
#endif
__host__ __device__ constexpr bool scan2_qpair(int d, int E) { return d >= S2_QPAIR_DIM && E <= S2_QPAIR_MAXE; }

// Row of a query pair in shared memory (scan2_qpair): per dimension the
// coordinates of queries 2p and 2p + 1 side by side, then their thresholds,
// then their sorted positions, padded to a multiple of 4 floats.
__host__ __device__ constexpr int qpair_row_floats(int d) { return (2 * (d + 2) + 3) & ~3; }
__host__ __device__ constexpr int qpair_floats(int d, int QM, int E)
{
    return scan2_qpair(d, E) ? (QM / 2) * qpair_row_floats(d) : 0;
}

// Entries of the per-warp histogram: the radix select of buffers of more
// than 64 entries needs 256 bins; the exact tail parks one id per buffer
// slot there.  With 64-entry buffers the parking shares the squared face-gap
// table instead when that is large enough (it is free once the scan is
// done), which leaves the histogram out.
__host__ __device__ constexpr bool hist_aliased(int d, int QM, int E) { return E <= 2 && 3 * d * QM >= 32 * E; }
__host__ __device__ constexpr int hist_entries(int d, int QM, int E)
{
    return hist_aliased(d, QM, E) ? 0 : (E <= 2 ? 32 * E : 256);
}

// Entries of the per-item table of neighbour key parts (even, so that what
// follows stays 16-byte aligned).
__host__ __device__ constexpr int dil_entries(int d) { return (3 * d + 1) & ~1; }

// Bytes of one warp's shared memory in k_scan2 (16-byte multiple):
// candidate buffers [QM][32E] u64, neighbour key parts [3d] u64, query rows
// [QM][QP] f32, query-pair rows [QM/2][QQ] f32 (scan2_qpair), cell-test
// thresholds [QM] f32, counts and sorted positions [QM] x 2, histogram
// [hist_entries(d, QM, E)], squared face gaps [3d][QM] f32, certificate radii [QM]
// f32, the item's cell and the level's extent [2d] i32.
__host__ __device__ constexpr size_t scan2_warp_bytes(int d, int QM, int E)
{
    return ((size_t)QM * 32 * E * 8 + (size_t)dil_entries(d) * 8 + (size_t)QM * query_row_floats(d) * 4 +
            (size_t)qpair_floats(d, QM, E) * 4 + (size_t)QM * 4 + (size_t)QM * 8 + (size_t)hist_entries(d, QM, E) * 4 +
            (size_t)QM * 3 * d * 4 + (size_t)QM * 4 + (size_t)2 * d * 4 + 15) &
           ~(size_t)15;
}

// Queries per work item for a candidate buffer of 32*E entries: 16 with the
// 64-entry buffers of K <= 32, 8 with larger ones (whose shared memory would
// otherwise hold an SM to 2 CTAs).
__host__ __device__ constexpr int scan2_queries_per_item(int E) { return E <= 2 ? 16 : 8; }

// Launch k_scan2 for dimension DIM with buffers of 32*E entries (E = 2, 4
// or 8) on stream s; mega selects the long-run walk that skips mega-tiles.
// Returns cudaSuccess or the launch error; *nofit is set (and nothing is
// launched) when the kernel cannot be resident on an SM.  *launches counts
// the launches made.
template <int DIM>
cudaError_t scan2_launch(const ScanArgs &a, int E, bool mega, size_t smem, cudaStream_t s, int nsm, int dev,
                         bool *nofit, int64_t *launches);

// The same for several joins at once: one launch of k_scan2_multi over the
// union queue in p (all jobs of dimension DIM and buffer size E).
template <int DIM>
cudaError_t scan2_launch_multi(const MultiScanArgs &p, int E, bool mega, size_t smem, cudaStream_t s, int nsm,
                               int dev, bool *nofit, int64_t *launches);

// Checked builds (KNN_CHECKS): the failed-check word of this unit's kernels
// (0 otherwise); clear = reset it to 0 after reading.
template <int DIM>
unsigned scan2_check_word(bool clear);

// Diagnostic builds (KNN_PHASE_TIMING): add this unit's phase cycles and
// event counts into out[0..32) (scan2_debug.cuh); reset = clear them.
template <int DIM>
cudaError_t scan2_debug_read(unsigned long long *out, bool reset);

}  // namespace knn
