// Tensor-core forms with 1 term on clusters of R CTAs (arXiv 1702.04728, Sec. 3
// and Sec. 3.1).
//
// The N-S stage is a DFT over rows of the zero-padded 512-point transform,
// evaluated on tcgen05 as X[m][t] = sum_k A[m][k] B[k][t] with A[m][2n] = cos,
// A[m][2n+1] = sin (2 pi n k_m / 512) and B holding the E-W phased feed line
// y_j of block time t as (yr, yi) in column t and (yi, -yr) in column 128 + t
// (FP16 operands, FP32 accumulation; one term: A and B rounded to FP16 once).
//   * R = 2 (BF_TC_DFT256_X1): the rows are the 256 clamped bins k_m = L(m)
//     of Eq. (1), one per N-S beam, so TMEM lane m of the pair is beam m;
//   * R = 4 (BF_TC_DFT512): the rows are all 512 bins k_m = m, the full
//     zero-padded transform (the 512 redundant beams of Sec. 3.1, twice the
//     GEMM and up-channel work), and the clamp of Eq. (1) is applied at the
//     output: bin k goes to every beam m with L(m) = k (none, one, or several
//     where aliasing maps pointings to one bin).
//
// A cluster of R CTAs owns a work item (channel segment, frame F, E-W beam
// j) and its six passes (3 blocks x 2 pols).  CTA r takes the rows
// 128 r .. 128 r + 127:
//   * its 128 rows of A for all K (128 KB) stay resident in shared memory,
//     reloaded only when the item's channel changes (R = 2; the 512-row
//     matrix does not depend on the frequency);
//   * each CTA builds 1/R of every B chunk (block times (128/R) r ..
//     (128/R)(r + 1) - 1: unpack, E-W toward beam j, FP16) into its own
//     shared memory and sends that part to the other CTAs with CTA-to-CTA
//     bulk copies, so every CTA holds the whole chunk and issues M = 128 MMAs
//     on its own rows;
//   * the accumulator of a pass is 128 bins x 256 columns, half of tensor
//     memory, so two passes alternate between the halves: the MMAs of pass
//     p + 1 overlap the up-channel passes (Sec. 3.2) of pass p.
// Warps: 0-7 build B (one (time, feed octet) task per thread and chunk for
// R = 2, half an octet for R = 4; the raw words of the next chunk prefetched
// into registers), 8-11 (one per tensor-memory lane quarter) run the
// up-channel passes and detection for one row each, warp 12 issues the MMAs
// and the A copies.  Hand-offs are mbarriers only (each builder warp sends the
// blocks it wrote to the other CTAs itself, so the builder warps never wait for
// one another); every wait is bounded by
// %globaltimer, and on expiry the CTA records the failure and leaves its loops
// (the other CTAs' waits then expire too).
#include "device_common.cuh"

#include <cuda_fp16.h>

#include <cstdint>
#include <mutex>

namespace chimebf {
namespace {

constexpr int kQKC = 64;                          // K elements (FP16) per chunk
constexpr int kQNCH = 2 * kFeed / kQKC;           // 8 chunks per pass
constexpr int kQSBO = kQKC / 8 * 128;             // 1024 bytes between 8-row groups of an operand
constexpr int kQAChunk = 128 * kQKC * 2;          // 16 KB: this CTA's 128 rows of A for one chunk
constexpr int kQBStage = 256 * kQKC * 2;          // 32 KB: one B chunk (N = 256)
constexpr int kQNB = 3;                           // B ring stages (225 KB of shared memory in all)
constexpr int kQBuild = 8;                        // builder warps (a multiple of 4)
constexpr int kQUp = 4;                           // up-channel warps
constexpr int kQThreads = 32 * (kQBuild + kQUp + 1);
constexpr int kQMmaWarp = kQBuild + kQUp;
// Register split (setmaxnreg): builders kQRegBuild, up-channel warps kQRegUp, the MMA warp
// keeps the launch count L; 8 x 104 + 4 x 176 + L <= 13 L needs L >= 128, which the
// launcher checks (with fewer, the up-channel warps' increase could never be granted).
constexpr int kQRegBuild = 104, kQRegUp = 176;
constexpr int kQRegLaunchMin = (kQBuild * kQRegBuild + kQUp * kQRegUp + 11) / 12;
// barriers: bfull[kQNB] bempty[kQNB] accfull[2] tfree[2] afull adone
constexpr int kQBars = 2 * kQNB + 6;
constexpr size_t kQSmemA = (size_t)kQNCH * kQAChunk;          // 128 KB
constexpr size_t kQSmemB = (size_t)kQNB * kQBStage;
constexpr size_t kQSmemTw = 8 * 8 * 16;
constexpr size_t kQSmem = kQSmemA + kQSmemB + kQSmemTw + 8 * kQBars;

// instruction descriptor: kind::f16, A = B = F16, D = F32, both K-major, M = 128, N = 256
constexpr uint32_t kQIdesc = (1u << 4) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint64_t qdesc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((128u >> 4) & 0x3FFF) << 16) |
           ((uint64_t)(((uint32_t)kQSBO >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ void qmma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(dtmem), "l"(adesc), "l"(bdesc), "r"(kQIdesc), "r"(accum)
        : "memory");
}

// commit of this thread's outstanding MMAs to the same mbarrier in every CTA of the cluster
template <int R>
__device__ __forceinline__ void qcommit_all(uint32_t mbar) {
    const uint16_t mask = (uint16_t)((1u << R) - 1u);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
                 :: "r"(mbar), "h"(mask) : "memory");
}

__device__ __forceinline__ void qcommit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t n_clusters() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}

// another CTA's shared-memory address of a local one
__device__ __forceinline__ uint32_t peer_addr(uint32_t a, uint32_t peer) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(peer));
    return r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void q_expect(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes) : "memory");
}

// bulk copy global -> this CTA's shared memory
__device__ __forceinline__ void q_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

// bulk copy this CTA's shared memory -> another CTA's (destination and its mbarrier
// as shared::cluster addresses), completing on that CTA's mbarrier
__device__ __forceinline__ void q_s2peer(uint32_t dst_cluster, uint32_t src_cta, uint32_t bytes,
                                         uint32_t mbar_cluster) {
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst_cluster), "r"(src_cta), "r"(bytes), "r"(mbar_cluster) : "memory");
}

__device__ __forceinline__ uint32_t qh2u(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }

// Byte offset of (row r, k-group kg) in a K-major chunk: 8 x 16-byte core matrices,
// k-groups 128 B apart, 8-row groups kQSBO apart.
__device__ __forceinline__ int qoff(int r, int kg) { return (r >> 3) * kQSBO + kg * 128 + (r & 7) * 16; }

// A builder thread's task of a chunk: block time t, feed octet `oct` and, for R = 4,
// which half of the octet (feeds 4 half .. 4 half + 3; R = 2 takes both halves).
// R = 2: lanes 0-7 take 8 consecutive times and lane bits 3-4 the octet; R = 4: lanes
// 0-7 the times, lane bit 3 the half, lane bit 4 and warp bit 0 the octet, so in both
// each warp load instruction reads whole 32-byte sectors.
template <int R>
__device__ __forceinline__ void q_task(uint32_t rank, int bt_id, int& t, int& oct, int& half) {
    const int lane = bt_id & 31, warp = bt_id >> 5;
    if constexpr (R == 2) {
        oct = (lane >> 3) & 3;
        half = 0;
        t = 64 * (int)rank + (lane & 7) + 8 * warp;
    } else {
        half = (lane >> 3) & 1;
        oct = ((warp & 1) << 1) | ((lane >> 4) & 1);
        t = 32 * (int)rank + (lane & 7) + 8 * (warp >> 1);
    }
}

template <int R>
struct QRaw;
template <>
struct QRaw<2> {
    uint4 v[kCyl];
};
template <>
struct QRaw<4> {
    uint2 v[kCyl];
};

template <int R>
__device__ __forceinline__ void q_load(const Seg& sg, long long row0, int kc, uint32_t rank, int bt_id, QRaw<R>& r) {
    int t, oct, half;
    q_task<R>(rank, bt_id, t, oct, half);
    const uint8_t* rp = frame_row(sg, row0 + t) + 2 * ((kQKC / 2) * kc + 8 * oct) + 8 * half;
#pragma unroll
    for (int c = 0; c < kCyl; ++c) {
        if constexpr (R == 2)
            r.v[c] = __ldg(reinterpret_cast<const uint4*>(rp + c * (kFeed * kPol)));
        else
            r.v[c] = __ldg(reinterpret_cast<const uint2*>(rp + c * (kFeed * kPol)));
    }
}

// unpack, E-W toward beam j, FP16 of feeds 4 h .. 4 h + 3 of an octet from the raw words
// (w0[c], w1[c]); row t = (yr, yi) per feed, row 128 + t = (yi, -yr)
__device__ __forceinline__ void q_build_half(const uint32_t (&w0)[kCyl], const uint32_t (&w1)[kCyl], uint32_t sel,
                                             const EwW& w, unsigned char* stage, int t, int kg) {
    cp y0, y1;                                    // SoA: (n, n + 2) and (n + 1, n + 3)
#pragma unroll
    for (int c = 0; c < kCyl; ++c) {
        const uint32_t g0 = __byte_perm(w0[c], 0u, sel), g1 = __byte_perm(w1[c], 0u, sel);
        const float2 xi0 = nib2<0>(g0, g1), xr0 = nib2<1>(g0, g1);
        const float2 xi1 = nib2<2>(g0, g1), xr1 = nib2<3>(g0, g1);
        if (c == 0) {
            y0 = {xr0, xi0};
            y1 = {xr1, xi1};
        } else {
            y0.re = fma2(xi0, w.NI[c - 1], fma2(xr0, w.R[c - 1], y0.re));
            y0.im = fma2(xr0, w.I[c - 1], fma2(xi0, w.R[c - 1], y0.im));
            y1.re = fma2(xi1, w.NI[c - 1], fma2(xr1, w.R[c - 1], y1.re));
            y1.im = fma2(xr1, w.I[c - 1], fma2(xi1, w.R[c - 1], y1.im));
        }
    }
    const float yr[4] = {y0.re.x, y1.re.x, y0.re.y, y1.re.y};
    const float yi[4] = {y0.im.x, y1.im.x, y0.im.y, y1.im.y};
    uint32_t vre[4], vim[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        vre[f] = qh2u(__floats2half2_rn(yr[f], yi[f]));
        vim[f] = qh2u(__floats2half2_rn(yi[f], -yr[f]));
    }
    *reinterpret_cast<uint4*>(stage + qoff(t, kg)) = make_uint4(vre[0], vre[1], vre[2], vre[3]);
    *reinterpret_cast<uint4*>(stage + qoff(128 + t, kg)) = make_uint4(vim[0], vim[1], vim[2], vim[3]);
}

template <int R>
__device__ __forceinline__ void q_build(const QRaw<R>& r, uint32_t sel, const EwW& w, unsigned char* stage,
                                        uint32_t rank, int bt_id) {
    int t, oct, half;
    q_task<R>(rank, bt_id, t, oct, half);
    if constexpr (R == 2) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t w0[kCyl], w1[kCyl];
#pragma unroll
            for (int c = 0; c < kCyl; ++c) {
                w0[c] = h ? r.v[c].z : r.v[c].x;
                w1[c] = h ? r.v[c].w : r.v[c].y;
            }
            q_build_half(w0, w1, sel, w, stage, t, 2 * oct + h);
        }
    } else {
        uint32_t w0[kCyl], w1[kCyl];
#pragma unroll
        for (int c = 0; c < kCyl; ++c) {
            w0[c] = r.v[c].x;
            w1[c] = r.v[c].y;
        }
        q_build_half(w0, w1, sel, w, stage, t, 2 * oct + half);
    }
}

// kStall: failure-detection check; the MMA thread stays idle, so no stage is ever released and
// every other wait runs out against the launch's bound.
template <int R, bool kStall>
__global__ void __launch_bounds__(kQThreads, 1) fused_tc_pair_kernel(const __grid_constant__ Batch bt) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;
    // [8 chunks][128 rows x 64 K] twiddles at 0, then the B ring, the pass-1 twiddles, mbarriers
    unsigned char* b_ring = smem + kQSmemA;                          // 2 x [256 rows x 64 K]
    float4* tw_s = reinterpret_cast<float4*>(b_ring + kQSmemB);
    uint64_t* mbar_s = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(tw_s) + kQSmemTw);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = cluster_rank();
    const uint32_t smem0 = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    const uint32_t bar0 = static_cast<uint32_t>(__cvta_generic_to_shared(&mbar_s[0]));
    auto bfull = [&](int s) { return bar0 + 8u * (uint32_t)s; };               // 8 builder warps + the others' parts
    auto bempty = [&](int s) { return bar0 + 8u * (uint32_t)(kQNB + s); };     // every CTA's MMA commit
    auto accfull = [&](int b) { return bar0 + 8u * (uint32_t)(2 * kQNB + b); }; // last commit of a pass
    auto tfree = [&](int b) { return bar0 + 8u * (uint32_t)(2 * kQNB + 2 + b); }; // the up-channel warps
    const uint32_t afull = bar0 + 8u * (uint32_t)(2 * kQNB + 4), adone = afull + 8u;

    if (warp == 0) {
        const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(&tmem_base_s));
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(dst) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < kQNB; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bfull(i)), "n"(kQBuild) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bempty(i)), "n"(R) : "memory");
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(accfull(i)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(tfree(i)), "n"(kQUp) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(afull) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(adone) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
    }
    for (int i = tid; i < 64; i += kQThreads) {
        const int it = i >> 3, c = i & 7;
        const float2 w0 = bt.tw128[(2 * it * c) & (kUp - 1)];
        const float2 w1 = bt.tw128[((2 * it + 1) * c) & (kUp - 1)];
        tw_s[i] = make_float4(w0.x, w1.x, w0.y, w1.y);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    cluster_sync();                        // every CTA's barriers exist before any remote arrival
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_s;
    constexpr int PASSES = kTds * kPol;
    const unsigned long long wlim = bt.wait_ns ? bt.wait_ns : kWaitNs;
    const int pair = (int)cluster_id(), npairs = (int)n_clusters();
    const int n_mine = bt.n_items > pair ? (bt.n_items - 1 - pair) / npairs + 1 : 0;
    auto item_of = [&](int k) { return pair + k * npairs; };

    if (warp == kQMmaWarp) {
        // ------------------------------ MMA / copy thread ------------------------------
        if (lane == 0 && !kStall) {
            uint32_t p_bfull = 0, p_tfree = 0, p_afull = 0, p_adone = 0;
            const unsigned char* a_cur = nullptr;
            long long c = 0, pass = 0;
            bool ok = true;
            int seg_cursor = 0;
            for (int k = 0; k < n_mine && ok; ++k) {
                const int item = item_of(k);
                while (seg_cursor + 1 < bt.n_segs && bt.segs[seg_cursor + 1].item_begin <= item) ++seg_cursor;
                const unsigned char* a_img = bt.segs[seg_cursor].a_img;
                if (a_img != a_cur) {
                    if (a_cur) {
                        // the MMAs that read the old twiddles are complete before they are replaced
                        qcommit(adone);
                        if (!mbar_wait(adone, p_adone, wlim)) ok = false;
                        p_adone ^= 1u;
                    }
                    q_expect(afull, (uint32_t)kQSmemA);
#pragma unroll 1
                    for (int kc = 0; kc < kQNCH; ++kc)
                        q_g2s(smem0 + (uint32_t)(kc * kQAChunk), a_img + (size_t)kc * (R * kQAChunk) + rank * kQAChunk,
                              (uint32_t)kQAChunk, afull);
                    if (!mbar_wait(afull, p_afull, wlim)) ok = false;
                    p_afull ^= 1u;
                    a_cur = a_img;
                }
                for (int ps = 0; ps < PASSES && ok; ++ps, ++pass) {
                    const int buf = (int)(pass & 1);
                    for (int kc = 0; kc < kQNCH && ok; ++kc, ++c) {
                        const int s = (int)(c % kQNB);
                        if (kc == 0 && pass >= 2) {
                            // the up-channel warps have read this accumulator half (pass - 2)
                            if (!mbar_wait(tfree(buf), (p_tfree >> buf) & 1u, wlim)) ok = false;
                            p_tfree ^= 1u << buf;
                        }
                        if (!mbar_wait(bfull(s), (p_bfull >> s) & 1u, wlim)) ok = false;
                        p_bfull ^= 1u << s;
                        if (!ok) break;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t a0 = smem0 + (uint32_t)(kc * kQAChunk);
                        const uint32_t b0 = smem0 + (uint32_t)(kQSmemA + s * kQBStage);
#pragma unroll
                        for (int ks = 0; ks < kQKC / 16; ++ks)
                            qmma(tmem + 256u * (uint32_t)buf, qdesc(a0 + ks * 256), qdesc(b0 + ks * 256),
                                 (kc | ks) ? 1u : 0u);
                        qcommit_all<R>(bempty(s));
                        if (kc == kQNCH - 1) qcommit(accfull(buf));
                        if (abort_s) ok = false;
                    }
                }
            }
            // every issued MMA is complete before the tensor memory is released
            qcommit(adone);
            if (!mbar_wait(adone, p_adone, wlim)) ok = false;
            if (!ok) abort_s = 1;
        }
        __syncwarp();
    } else if (warp < kQBuild) {
        // ------------------------------ builders ------------------------------
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" :: "n"(kQRegBuild) : "memory");
        const int bt_id = tid;                                       // 0 .. 127
        uint32_t p_bempty = 0;
        long long c = 0;
        bool ok = true;
        for (int k = 0; k < n_mine && ok; ++k) {
            const int item = item_of(k);
            int sgi = 0;
            while (sgi + 1 < bt.n_segs && bt.segs[sgi + 1].item_begin <= item) ++sgi;
            const Seg& sg = bt.segs[sgi];
            const int local = item - sg.item_begin;
            const int F = local >> 2, j = local & 3;
            EwW w;
            load_ew_frame(sg, bt.ew, F, j, w);
            QRaw<R> raw;
            q_load<R>(sg, (long long)F * kFrame, 0, rank, bt_id, raw);
            for (int ps = 0; ps < PASSES && ok; ++ps) {
                const int blk = ps >> 1, pol = ps & 1;
                const uint32_t sel = 0x4400u | ((2u + pol) << 4) | (uint32_t)pol;
                for (int kc = 0; kc < kQNCH && ok; ++kc, ++c) {
                    const int s = (int)(c % kQNB);
                    if (c >= kQNB) {
                        // every CTA's MMAs have read stage s (chunk c - kQNB), and with them the
                        // copies out of it into the other CTAs
                        if (!mbar_wait(bempty(s), (p_bempty >> s) & 1u, wlim)) ok = false;
                        p_bempty ^= 1u << s;
                    }
                    QRaw<R> cur = raw;
                    const bool last = kc + 1 == kQNCH;
                    if (!last || ps + 1 < PASSES) {
                        const int nblk = last ? ((ps + 1) >> 1) : blk;
                        q_load<R>(sg, (long long)F * kFrame + nblk * kUp, last ? 0 : kc + 1, rank, bt_id, raw);
                    }
                    unsigned char* stage = b_ring + s * kQBStage;
                    q_build<R>(cur, sel, w, stage, rank, bt_id);
                    // the generic-proxy stores are visible to the tensor core and the bulk copies
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    // the warp stops as one (an expired wait in any lane, or elsewhere in the CTA)
                    if (__any_sync(0xffffffffu, !ok || abort_s != 0)) {
                        ok = false;
                        break;
                    }
                    if (lane == 0) {
                        // the warp wrote one contiguous block of every 8-row group it touched (a whole
                        // 1 KB group for R = 2, half of one for R = 4) at rows t and 128 + t: it sends
                        // them to the other CTAs itself, so no barrier holds the builders together
                        const uint32_t st = smem0 + (uint32_t)(kQSmemA + s * kQBStage);
                        uint32_t o0, len;
                        if constexpr (R == 2) {
                            o0 = (8u * rank + (uint32_t)warp) * (uint32_t)kQSBO;
                            len = (uint32_t)kQSBO;
                        } else {
                            o0 = (4u * rank + (uint32_t)(warp >> 1)) * (uint32_t)kQSBO + (uint32_t)(warp & 1) * (kQSBO / 2);
                            len = (uint32_t)kQSBO / 2;
                        }
                        const uint32_t o1 = o0 + 16u * (uint32_t)kQSBO;
                        q_expect(bfull(s), 2u * (R - 1) * len);   // the same warp of each other CTA sends as much
#pragma unroll
                        for (uint32_t d = 1; d < (uint32_t)R; ++d) {
                            const uint32_t peer = (rank + d) % (uint32_t)R;
                            const uint32_t pbar = peer_addr(bfull(s), peer);
                            q_s2peer(peer_addr(st + o0, peer), st + o0, len, pbar);
                            q_s2peer(peer_addr(st + o1, peer), st + o1, len, pbar);
                        }
                    }
                }
            }
        }
        if (!ok) abort_s = 1;
    } else {
        // ------------------------------ up-channel warps ------------------------------
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" :: "n"(kQRegUp) : "memory");
        const int q4 = warp & 3;                                   // tensor-memory lane quarter
        const int ell = 32 * q4 + lane;                            // this thread's row: 128 rank + ell
        uint32_t p_acc = 0;
        long long pass = 0;
        bool ok = true;
        for (int k = 0; k < n_mine && ok; ++k) {
            const int item = item_of(k);
            int sgi = 0;
            while (sgi + 1 < bt.n_segs && bt.segs[sgi + 1].item_begin <= item) ++sgi;
            const Seg& sg = bt.segs[sgi];
            const int local = item - sg.item_begin;
            const int F = local >> 2, j = local & 3;
            float2 acc[kSub];
#pragma unroll
            for (int q = 0; q < kSub; ++q) acc[q] = make_float2(0.f, 0.f);
            for (int ps = 0; ps < PASSES && ok; ++ps, ++pass) {
                const int buf = (int)(pass & 1);
                if (!mbar_wait(accfull(buf), (p_acc >> buf) & 1u, wlim)) ok = false;
                p_acc ^= 1u << buf;
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t base = tmem + (static_cast<uint32_t>(32 * q4) << 16) + 256u * (uint32_t)buf;
                upchan_pass1_split(base, tw_s, 0, 1);
                tmem_wait_st();
                upchan_pass2_split(base, acc, nullptr, 0, 1);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(tfree(buf));
                if (abort_s) ok = false;
            }
            if (ok) {
                if constexpr (R == 2) {
                    float* o = sg.out + (long long)(kNs * j + 128 * (int)rank + ell) * sg.beam_stride + F;
#pragma unroll
                    for (int q = 0; q < kSub; ++q) o[(long long)q * sg.sub_stride] = acc[q].x + acc[q].y;
                } else {
                    // the clamp (Eq. 1): bin 128 r + ell feeds every beam m with L(m) = that bin
                    const int16_t* inv = bt.inv + (size_t)sg.table * kInvLen;
                    for (int m = inv[128 * (int)rank + ell]; m >= 0; m = inv[kBins + m]) {
                        float* o = sg.out + (long long)(kNs * j + m) * sg.beam_stride + F;
#pragma unroll
                        for (int q = 0; q < kSub; ++q) o[(long long)q * sg.sub_stride] = acc[q].x + acc[q].y;
                    }
                }
            }
        }
        if (!ok) abort_s = 1;
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // every CTA of the cluster is done issuing copies; in a run that completed, each CTA's MMA
    // thread has also seen every copy into it land (its last "B full" waits)
    cluster_sync();
    if (abort_s) {
        if (tid == 0 && bt.status) atomicExch(bt.status, 1);
        if (warp == 0) {
            // after an expired wait, copies that another CTA issued before the cluster barrier
            // may still be landing in this CTA's shared memory: warp 0 keeps the CTA resident
            // a while (bounded), then reconverges for the TMEM release
            const unsigned long long t0 = globaltimer();
            while (globaltimer() - t0 < 200000ull) {
            }
            __syncwarp();
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tmem) : "memory");
    }
}

// Launch of the R-CTA cluster kernel; grid is a multiple of R.
template <int R, bool kStall = false>
cudaError_t cluster_launch(const Batch& b, int grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kQThreads);
    cfg.dynamicSmemBytes = kQSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = R;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, fused_tc_pair_kernel<R, kStall>, b);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Once per device and cluster size: the register split must fit in what the kernel was
// launched with (else the up-channel warps' increase could never be granted: such a build
// is refused), the shared-memory size is set, and the clusters that fit at once are counted.
template <int R, bool kStall = false>
cudaError_t cluster_setup(int* max_clusters) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    static std::once_flag once[kMaxDevices];
    static cudaError_t result[kMaxDevices];
    static int clusters[kMaxDevices];
    std::call_once(once[dev], [&] {
        cudaFuncAttributes fa;
        cudaError_t r = cudaFuncGetAttributes(&fa, fused_tc_pair_kernel<R, kStall>);
        if (r == cudaSuccess && fa.numRegs < kQRegLaunchMin) r = cudaErrorInvalidConfiguration;
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(fused_tc_pair_kernel<R, kStall>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kQSmem);
        int sms = 0;
        if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int n = sms / R;
        if (r == cudaSuccess && R > 2) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)(R * n));
            cfg.blockDim = dim3(kQThreads);
            cfg.dynamicSmemBytes = kQSmem;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = R;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            r = cudaOccupancyMaxActiveClusters(&n, fused_tc_pair_kernel<R, kStall>, &cfg);
        }
        clusters[dev] = n;
        result[dev] = r;
    });
    *max_clusters = clusters[dev];
    return result[dev];
}

}  // namespace

cudaError_t fused_tc_pair_launch(const Batch& b, int grid, cudaStream_t s) {
    if (b.n_items <= 0) return cudaSuccess;
    grid &= ~1;
    if (grid < 2) grid = 2;
    int max_clusters = 0;
    cudaError_t e = cluster_setup<2>(&max_clusters);
    if (e != cudaSuccess) return e;
    return cluster_launch<2>(b, grid, s);
}

cudaError_t fused_tc_dft512_launch(const Batch& b, cudaStream_t s) {
    if (b.n_items <= 0) return cudaSuccess;
    int max_clusters = 0;
    cudaError_t e = cluster_setup<4>(&max_clusters);
    if (e != cudaSuccess) return e;
    if (max_clusters < 1) return cudaErrorInvalidConfiguration;
    return cluster_launch<4>(b, 4 * std::min(max_clusters, b.n_items), s);
}

cudaError_t fused_tc_pair_stall_launch(const Batch& b, int cluster, cudaStream_t s) {
    if (b.n_items <= 0) return cudaSuccess;
    int max_clusters = 0;
    cudaError_t e = cluster == 4 ? cluster_setup<4, true>(&max_clusters) : cluster_setup<2, true>(&max_clusters);
    if (e != cudaSuccess) return e;
    return cluster == 4 ? cluster_launch<4, true>(b, 4, s) : cluster_launch<2, true>(b, 2, s);
}

}  // namespace chimebf
