// stage_tab.cuh -- the table of stage-kernel instances: nf stage derivatives
// read (0..7), nh demag sources (1: the exact field, or p + 1 = 1..7 history
// fields), last stage or not; stage 0 (input m0, at most ABM2's one
// derivative, the exact field) has its own two instances.
#pragma once
#include "kernels_impl.cuh"

namespace {

template <typename T, int NF, int NH> const void *stage_k(bool last, bool stage0)
{
    if (stage0) {
        if constexpr (NH == 1 && NF <= 1) return last ? nullptr : (const void *)k_stage<T, NF, NH, false, true>;
        return nullptr;
    }
    return last ? (const void *)k_stage<T, NF, NH, true, false> : (const void *)k_stage<T, NF, NH, false, false>;
}

template <typename T, int NF> const void *stage_nh(int nh, bool last, bool stage0)
{
    switch (nh) {
    case 1: return stage_k<T, NF, 1>(last, stage0);
    case 2: return stage_k<T, NF, 2>(last, stage0);
    case 3: return stage_k<T, NF, 3>(last, stage0);
    case 4: return stage_k<T, NF, 4>(last, stage0);
    case 5: return stage_k<T, NF, 5>(last, stage0);
    case 6: return stage_k<T, NF, 6>(last, stage0);
    case 7: return stage_k<T, NF, 7>(last, stage0);
    }
    return nullptr;
}

template <typename T> const void *stage_tab(int nf, int nh, bool last, bool stage0)
{
    switch (nf) {
    case 0: return stage_nh<T, 0>(nh, last, stage0);
    case 1: return stage_nh<T, 1>(nh, last, stage0);
    case 2: return stage_nh<T, 2>(nh, last, stage0);
    case 3: return stage_nh<T, 3>(nh, last, stage0);
    case 4: return stage_nh<T, 4>(nh, last, stage0);
    case 5: return stage_nh<T, 5>(nh, last, stage0);
    case 6: return stage_nh<T, 6>(nh, last, stage0);
    case 7: return stage_nh<T, 7>(nh, last, stage0);
    }
    return nullptr;
}

}  // namespace
