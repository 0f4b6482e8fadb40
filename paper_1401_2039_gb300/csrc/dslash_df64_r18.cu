// Hopping-term kernel in double-float arithmetic with double-float storage
// and 18-real links: the residuals r = b - M x of the reliable updates
// (the loop over the hops is df_hops, dslash_df.cuh).
#include "dslash_df.cuh"

namespace wd {
namespace {

// STAGE: each hop's link record is copied into shared memory by cp.async
// while the previous hop computes (df_hops)
template <int DAG, int EPI, int NORM, int BLOCK, int MINB, int STAGE>
__global__ void __launch_bounds__(BLOCK, MINB) k_dslash_df(const DslashArgs<df64> a) {
    df64 nrm[1] = {df64(0.0f, 0.0f)};
    const long h = a.h0 + (long)blockIdx.x * BLOCK + threadIdx.x;
    if (h < a.h1) {
        int c[4];
        site_coords(a.g, h, a.parity, c);
        dfl acc[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) acc[k] = 0;
        if constexpr (STAGE) {
            __shared__ uint4 stage[2 * DF_LINK_PLANES * BLOCK];
            df_hops<DAG, BLOCK>(a.g, a.gauge_out, a.gauge_in, a.dir_bytes, a.ph, a.in, a.g.stride,
                                1, 0, h, c, acc, stage, a.phase_on);
        } else {
            df_hops<DAG>(a.g, a.gauge_out, a.gauge_in, a.dir_bytes, a.ph, a.in, a.g.stride, 1, 0,
                         h, c, acc, nullptr, a.phase_on);
        }
        df64 o[24];
        if (EPI == EPI_XPAY) {
            df64 xv[24];
            Rec<df64, 24>::template load<df64, 0>(a.x, a.g.stride, h, xv);
            if (a.twist_on) twist_site(xv, a.twist);
#pragma unroll
            for (int k = 0; k < 24; ++k) o[k] = settle(xv[k] + a.scale * acc[k]);
        } else {
#pragma unroll
            for (int k = 0; k < 24; ++k) o[k] = settle(a.scale * acc[k]);
            if (a.twist_on) twist_site(o, -a.twist);
        }
        Rec<df64, 24>::store(a.out, a.g.stride, h, o);
        if (NORM) {
            df64 sq = 0;
#pragma unroll
            for (int k = 0; k < 24; ++k) sq += o[k] * o[k];
            nrm[0] = sq;
        }
    }
    if (NORM) warp_partials<BLOCK, 1>(nrm, a.g.vh, a.red.partials);
}

template <int DAG, int EPI, int NORM, int CFG>
void launch_df(const DslashArgs<df64> &a, cudaStream_t s) {
    constexpr DslashCfg C = DSLASH_DF_CFGS[CFG];
    const unsigned grid = (unsigned)((a.h1 - a.h0 + C.block - 1) / C.block);
    k_dslash_df<DAG, EPI, NORM, C.block, C.minb, C.stage><<<grid, C.block, 0, s>>>(a);
}

template <int DAG, int EPI>
void launch_df_cfg(int cfg, const DslashArgs<df64> &a, cudaStream_t s) {
    switch (cfg) {
    case 1: launch_df<DAG, EPI, 0, 1>(a, s); break;
    case 2: launch_df<DAG, EPI, 0, 2>(a, s); break;
    case 3: launch_df<DAG, EPI, 0, 3>(a, s); break;
    case 4: launch_df<DAG, EPI, 0, 4>(a, s); break;
    case 5: launch_df<DAG, EPI, 0, 5>(a, s); break;
    case 6: launch_df<DAG, EPI, 0, 6>(a, s); break;
    case 7: launch_df<DAG, EPI, 0, 7>(a, s); break;
    default: launch_df<DAG, EPI, 0, 0>(a, s); break;
    }
}

}  // namespace

cudaError_t launch_dslash_df64_r18(const DslashLaunch &L, cudaStream_t s) {
    DslashArgs<df64> a;
    a.g = L.g;
    a.gauge_out = (const char *)L.gauge->ptr[L.out_parity];
    a.gauge_in = (const char *)L.gauge->ptr[1 - L.out_parity];
    a.dir_bytes = L.gauge->dir_bytes;
    a.out = L.out;
    a.in = L.in;
    a.x = L.x;
    a.scale = df64(L.scale);
    for (int i = 0; i < 8; ++i) a.ph[i] = df64(L.phase[i]);
    a.phase_on = phase_mask(L.phase);
    a.parity = L.out_parity;
    a.red = L.red ? *L.red : Reduction{nullptr, nullptr, nullptr, FIN_NONE};
    a.twist = df64(L.twist);
    a.twist_on = L.twist != 0.0;
    a.h0 = L.h_begin;
    a.h1 = L.h_end < 0 ? L.g.vh : L.h_end;
    if (a.h0 < 0 || a.h1 > L.g.vh || a.h0 > a.h1) return cudaErrorInvalidValue;
    if (a.h1 == a.h0) return cudaSuccess;
    if (L.red && (a.h0 != 0 || a.h1 != L.g.vh)) return cudaErrorInvalidValue;
    if (L.red) {   // fused norm; the residuals never use it: one configuration
        if (L.dagger) launch_df<1, EPI_XPAY, 1, 0>(a, s);
        else launch_df<0, EPI_XPAY, 1, 0>(a, s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_finish_partials(a.red, (L.g.vh + 31) / 32, s);
    } else if (L.epi == EPI_PLAIN) {
        if (L.dagger) launch_df_cfg<1, EPI_PLAIN>(L.cfg, a, s);
        else launch_df_cfg<0, EPI_PLAIN>(L.cfg, a, s);
    } else {
        if (L.dagger) launch_df_cfg<1, EPI_XPAY>(L.cfg, a, s);
        else launch_df_cfg<0, EPI_XPAY>(L.cfg, a, s);
    }
    return cudaGetLastError();
}

}  // namespace wd
