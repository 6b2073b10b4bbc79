// fft_pipe.cu -- instances of the pipelined large-mesh passes.
#include "kernels_impl.cuh"

const void *mmxk_tab_pipe(int kind, bool f64, int L)
{
    switch (kind) {
    case K_XFP: return f64 ? xfp_fn<double>(L) : xfp_fn<float>(L);
    case K_YFP: return f64 ? yfp_fn<double>(L) : yfp_fn<float>(L);
    case K_YIP: return f64 ? yip_fn<double>(L) : yip_fn<float>(L);
    case K_ZMP: return f64 ? zmp_fn<double>(L) : zmp_fn<float>(L);
    case K_XIT: return f64 ? nullptr : xit_fn<float>(L);
    case K_YF4: return f64 || L != 1024 ? nullptr : (const void *)k_yf4<float>;
    case K_YI4: return f64 || L != 1024 ? nullptr : (const void *)k_yi4<float>;
    case K_XF4: return f64 || L != 1024 ? nullptr : (const void *)k_xf4<float>;
    case K_XI4: return f64 || L != 1024 ? nullptr : (const void *)k_xi_t<float, 1024, true>;
    // K_XF4H: L = rows per item (16 or 8) of the 512-point pass
    case K_XF4H: return f64 ? nullptr : (L == 16 ? (const void *)k_xf4h<float, 16> : (L == 8 ? (const void *)k_xf4h<float, 8> : nullptr));
    case K_XI4H: return f64 || L != 512 ? nullptr : (const void *)k_xi_t<float, 512, true>;
    }
    return nullptr;
}
