// fft_split.cu -- instances of the split y / z passes (YF, ZM, YI).
#include "kernels_impl.cuh"

const void *mmxk_tab_split(int kind, bool f64, int L)
{
    switch (kind) {
    case K_YF: return f64 ? yf_fn<double>(L) : yf_fn<float>(L);
    case K_YI: return f64 ? yi_fn<double>(L) : yi_fn<float>(L);
    case K_ZM: return f64 ? zm_fn<double>(L) : zm_fn<float>(L);
    case K_ZMR: return f64 ? zmr_fn<double>(L) : zmr_fn<float>(L);
    }
    return nullptr;
}
