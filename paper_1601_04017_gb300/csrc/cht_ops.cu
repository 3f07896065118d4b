// Launchers of the batched probe kernels (see cht_ops.cuh).
#include <atomic>

#include "cht_ops.cuh"

namespace cht {
namespace {

// Launch with programmatic stream serialization (see pdl_enter).
template <typename K>
cudaError_t launch_pdl(K kernel, unsigned grid, unsigned block, size_t smem, cudaStream_t s, const OpArgs& a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}


template <int G, int V, int MODE, int kFlags = 0>
cudaError_t launch_one(const OpArgs& a, int ctas_per_sm, cudaStream_t s) {
    static std::atomic<int> occ{0};
    int per_sm = occ.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        cudaError_t e =
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, op_kernel<G, V, MODE, kFlags>, kOpBlock, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        occ.store(per_sm, std::memory_order_relaxed);
    }
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    u64 grid = u64(sm_count()) * u64(per_sm);
    const u64 need = (a.n + kOpBlock - 1) / kOpBlock;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    const cudaError_t e = launch_pdl(op_kernel<G, V, MODE, kFlags>, unsigned(grid), kOpBlock, 0, s, a);
    count_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Per-thread operations (group_width = -1), V = 2 or 4 cells per step.
template <int V, int MODE>
cudaError_t launch_thread_v(const OpArgs& a, int ctas_per_sm, cudaStream_t s) {
    static std::atomic<int> occ{0};
    int per_sm = occ.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        cudaError_t e =
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, thread_kernel<V, MODE>, kThreadBlock, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        occ.store(per_sm, std::memory_order_relaxed);
    }
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    u64 grid = u64(sm_count()) * u64(per_sm);
    const u64 need = (a.n + kThreadBlock - 1) / kThreadBlock;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    const cudaError_t e = launch_pdl(thread_kernel<V, MODE>, unsigned(grid), kThreadBlock, 0, s, a);
    count_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <int MODE>
cudaError_t launch_thread(const OpArgs& a, int v, int ctas_per_sm, cudaStream_t s) {
    return v == 2 ? launch_thread_v<2, MODE>(a, ctas_per_sm, s) : launch_thread_v<4, MODE>(a, ctas_per_sm, s);
}

// Tables with tombstone reuse or the full key space: kernels exist for the
// automatic windows only -- 1 lane x 1 sector, 2 lanes x 2 sectors, 4 lanes x
// 1 or 2 sectors; any other configured window takes the nearest of these.
template <int MODE, int F>
cudaError_t launch_window(const OpArgs& a, int g, int v, int ctas_per_sm, cudaStream_t s) {
    if (g <= 1) return launch_one<1, 2, MODE, F>(a, ctas_per_sm, s);
    if (g == 2) return launch_one<2, 4, MODE, F>(a, ctas_per_sm, s);
    if (g == 4 && v != 4) return launch_one<4, 2, MODE, F>(a, ctas_per_sm, s);
    return launch_one<4, 4, MODE, F>(a, ctas_per_sm, s);
}

template <int MODE>
cudaError_t launch_flagged(const OpArgs& a, int g, int v, int flags, int ctas_per_sm, cudaStream_t s) {
    constexpr bool fills = mode_fills(MODE);
    switch (flags) {
        case kFlagReuse:
            if constexpr (fills) return launch_window<MODE, kFlagReuse>(a, g, v, ctas_per_sm, s);
            break;
        case kFlagFullKeys: return launch_window<MODE, kFlagFullKeys>(a, g, v, ctas_per_sm, s);
        case kFlagReuse | kFlagFullKeys:
            if constexpr (fills) return launch_window<MODE, kFlagReuse | kFlagFullKeys>(a, g, v, ctas_per_sm, s);
            break;
        default: break;
    }
    return cudaErrorInvalidValue;
}

// (group width G, cells per lane V): G = 1 always loads a whole sector.
template <int MODE>
cudaError_t launch_mode(const OpArgs& a, int g, int v, int ctas_per_sm, cudaStream_t s) {
    const int flags = ((mode_fills(MODE) && a.reuse) ? kFlagReuse : 0) | (a.full_keys ? kFlagFullKeys : 0);
    if (g < 0) {
        // the per-thread kernels: plain tables, the whole batch in one
        // grid-stride pass (in-order pieces take the 1-lane group loop)
        if (!flags && a.chunk == 0) return launch_thread<MODE>(a, v, ctas_per_sm, s);
        g = 1;
        if (v != 4) v = 2;
    }
    if (flags) return launch_flagged<MODE>(a, g, v, flags, ctas_per_sm, s);
    if (v == 4) {
        switch (g) {
            case 1: return launch_one<1, 4, MODE>(a, ctas_per_sm, s);
            case 2: return launch_one<2, 4, MODE>(a, ctas_per_sm, s);
            case 4: return launch_one<4, 4, MODE>(a, ctas_per_sm, s);
            case 8: return launch_one<8, 4, MODE>(a, ctas_per_sm, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (v == 2) {
        switch (g) {
            case 1: return launch_one<1, 2, MODE>(a, ctas_per_sm, s);
            case 2: return launch_one<2, 2, MODE>(a, ctas_per_sm, s);
            case 4: return launch_one<4, 2, MODE>(a, ctas_per_sm, s);
            case 8: return launch_one<8, 2, MODE>(a, ctas_per_sm, s);
            case 16: return launch_one<16, 2, MODE>(a, ctas_per_sm, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (g) {
        case 1: return launch_one<1, 2, MODE>(a, ctas_per_sm, s);
        case 2: return launch_one<2, 1, MODE>(a, ctas_per_sm, s);
        case 4: return launch_one<4, 1, MODE>(a, ctas_per_sm, s);
        case 8: return launch_one<8, 1, MODE>(a, ctas_per_sm, s);
        case 16: return launch_one<16, 1, MODE>(a, ctas_per_sm, s);
        case 32: return launch_one<32, 1, MODE>(a, ctas_per_sm, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int MODE, int WD, bool RE, int BLOCK = kAggBlock>
cudaError_t launch_agg(const OpArgs& a, int ctas_per_sm, cudaStream_t s) {
    constexpr size_t smem = agg_smem_bytes<MODE, BLOCK>();
    static std::atomic<int> occ{0};
    int per_sm = occ.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(iou_agg_kernel<MODE, WD, RE, BLOCK>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        // as much of the unified L1 / shared memory as shared memory as the
        // kernel can use (38 KB per 256-thread CTA, 152 KB per 1024-thread CTA)
        e = cudaFuncSetAttribute(iou_agg_kernel<MODE, WD, RE, BLOCK>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 100);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, iou_agg_kernel<MODE, WD, RE, BLOCK>, BLOCK, smem);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        occ.store(per_sm, std::memory_order_relaxed);
    }
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    u64 grid = u64(sm_count()) * u64(per_sm);
    const u64 nwin = (a.n + 4 * BLOCK - 1) / (4 * BLOCK);
    if (grid > nwin) grid = nwin;
    if (grid < 1) grid = 1;
    const cudaError_t e = launch_pdl(iou_agg_kernel<MODE, WD, RE, BLOCK>, unsigned(grid), BLOCK, smem, s, a);
    count_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

cudaError_t launch_iou_aggregated(Mode mode, const OpArgs& a, bool warp_dedup, int ctas_per_sm, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    const bool re = a.reuse != 0;
    if (mode == kIouAdd) {
        if (re)
            return warp_dedup ? launch_agg<kIouAdd, 2, true>(a, ctas_per_sm, s)
                              : launch_agg<kIouAdd, 1, true>(a, ctas_per_sm, s);
        return warp_dedup ? launch_agg<kIouAdd, 2, false>(a, ctas_per_sm, s)
                          : launch_agg<kIouAdd, 1, false>(a, ctas_per_sm, s);
    }
    if (mode == kIouOverwrite) {
        if (re)
            return warp_dedup ? launch_agg<kIouOverwrite, 2, true>(a, ctas_per_sm, s)
                              : launch_agg<kIouOverwrite, 1, true>(a, ctas_per_sm, s);
        return warp_dedup ? launch_agg<kIouOverwrite, 2, false>(a, ctas_per_sm, s)
                          : launch_agg<kIouOverwrite, 1, false>(a, ctas_per_sm, s);
    }
    // update: equal keys fold the same way; no cell is filled, so neither the
    // warp pre-reduction nor tombstone reuse applies
    if (mode == kUpdAdd) return launch_agg<kUpdAdd, 0, false>(a, ctas_per_sm, s);
    if (mode == kUpdOverwrite) return launch_agg<kUpdOverwrite, 0, false>(a, ctas_per_sm, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_iou_aggregated_wide(Mode mode, const OpArgs& a, bool warp_dedup, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    const bool re = a.reuse != 0;
    if (mode == kIouAdd) {
        if (re)
            return warp_dedup ? launch_agg<kIouAdd, 2, true, 1024>(a, 0, s) : launch_agg<kIouAdd, 1, true, 1024>(a, 0, s);
        return warp_dedup ? launch_agg<kIouAdd, 2, false, 1024>(a, 0, s) : launch_agg<kIouAdd, 1, false, 1024>(a, 0, s);
    }
    if (mode == kIouOverwrite) {
        if (re)
            return warp_dedup ? launch_agg<kIouOverwrite, 2, true, 1024>(a, 0, s)
                              : launch_agg<kIouOverwrite, 1, true, 1024>(a, 0, s);
        return warp_dedup ? launch_agg<kIouOverwrite, 2, false, 1024>(a, 0, s)
                          : launch_agg<kIouOverwrite, 1, false, 1024>(a, 0, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_op(Mode mode, const OpArgs& a, int group_width, int lane_cells, int ctas_per_sm,
                      cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    const int v = lane_cells;
    switch (mode) {
        case kFind: return launch_mode<kFind>(a, group_width, v, ctas_per_sm, s);
        case kInsert: return launch_mode<kInsert>(a, group_width, v, ctas_per_sm, s);
        case kIouAdd: return launch_mode<kIouAdd>(a, group_width, v, ctas_per_sm, s);
        case kIouOverwrite: return launch_mode<kIouOverwrite>(a, group_width, v, ctas_per_sm, s);
        case kErase: return launch_mode<kErase>(a, group_width, v, ctas_per_sm, s);
        case kUpdAdd: return launch_mode<kUpdAdd>(a, group_width, v, ctas_per_sm, s);
        case kUpdOverwrite: return launch_mode<kUpdOverwrite>(a, group_width, v, ctas_per_sm, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cht
