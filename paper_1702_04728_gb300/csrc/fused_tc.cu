// Tensor-core form of the fan-beam path for sm_103a (arXiv 1702.04728, Sec. 3).
//
// Same work decomposition as the FP32 kernel -- one CTA per SM owns
// (channel segment, frame F, E-W beam j) and makes six passes (3 blocks x 2
// pols) -- but the N-S stage (Sec. 3.1: zero-padded FFT kept at the 256 bins
// of Eq. 1) is evaluated as the equivalent dense DFT over the clamped rows on
// the tcgen05 tensor cores:
//
//   X[m][t] = sum_n exp(-2 pi i n L(m) / 512) y_j[n][t],   m < 256, n < 256,
//
// with y_j the E-W phased feed line (Sec. 3) of block time t.  As a real GEMM:
// rows = bins m (two M = 128 tiles), columns = (t, re/im) (N = 256), K = (n,
// re/im) = 512.  With A[m][2n] = cos, A[m][2n+1] = sin (of 2 pi n L / 512) the
// column t of B holds (yr, yi) and column 128 + t holds (yi, -yr), so the two
// halves give Re and Im of X with one A.  The accumulator lands in tensor
// memory where the up-channel passes read it: lane = bin (m, m + 128), columns
// [0, 128) = Re X(t), [128, 256) = Im X(t) of each 256-column bin half.
//
// Precision: FP16 operands, FP32 accumulation.  y is split y = y_hi + y_lo in
// FP16 (22 bits together); the twiddles are FP16 (hi) and, for three terms,
// also lo.  Terms: 1 = A_hi y_hi, 2 = + A_hi y_lo, 3 = + A_lo y_hi.
//
// Pipeline per pass: K is streamed in chunks through two shared-memory stages.
// Thread 0 starts the bulk copy (TMA engine) of each twiddle chunk one chunk
// ahead; all warps build the B chunk (unpack, E-W, FP16 split) from raw bytes
// prefetched into registers one chunk ahead and arrive on the stage's "B full"
// mbarrier; thread 0 waits for B and twiddles, issues the MMAs and commits
// them to the stage's "empty" mbarrier, which the producers wait on before
// reusing the stage.  No CTA barrier sits inside the chunk loop.  Every wait is
// bounded by %globaltimer; on expiry the kernel records an error and leaves.
#include "device_common.cuh"

#include <cuda_fp16.h>

#include <cstdint>
#include <mutex>

namespace chimebf {
namespace {


template <int TERMS>
struct TcCfg {
    static constexpr int KC = TERMS == 3 ? 32 : 64;              // K elements (FP16) per chunk
    static constexpr int NCH = 2 * kFeed / KC;                    // chunks per pass
    static constexpr int SBO = KC / 8 * 128;                      // bytes between 8-row groups
    static constexpr int OPER = 256 * KC * 2;                     // bytes of one 256-row operand chunk
    static constexpr bool A_LO = TERMS == 3;
    static constexpr bool B_LO = TERMS >= 2;
    static constexpr int A_STAGE = OPER * (A_LO ? 2 : 1);         // twiddle ring stage
    static constexpr int B_STAGE = OPER * (B_LO ? 2 : 1);         // data ring stage
    static constexpr int NA = 2;                                  // twiddle ring depth (a smaller shared-memory
                                                                  // footprint leaves L1 for the raw loads)
    static constexpr int NOCT = KC / 16;                          // 8-feed octets per chunk
    static constexpr int NT = 288;                                // 8 producer warps + 1 MMA warp
    static constexpr int NPROD = 256;                             // producer threads
    static constexpr size_t SMEM = (size_t)NA * A_STAGE + 2ull * B_STAGE + 8 * 8 * 16 + 8 * (6 + 2 * NA);
};

// Byte offset of element (row r, k) in a K-major operand chunk without
// swizzle: 8 x 16-byte core matrices, k-groups 128 B apart, row groups SBO apart.
template <int SBO>
__device__ __forceinline__ int core_off(int r, int kgroup) {
    return (r >> 3) * SBO + kgroup * 128 + (r & 7) * 16;
}

// shared-memory matrix descriptor (no swizzle, version 1)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor: kind::f16, A = B = F16, D = F32, both K-major, M = 128, N = 256
constexpr uint32_t kIdesc = (1u << 4) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(dtmem), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ uint32_t h2u(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }

// Producer tasks (t, octet): 8 feeds x 2 pols of every cylinder, one 16-byte
// load each.  Lanes run over t so the B stores of a quarter warp fill one
// 128-byte line.
template <int TERMS>
struct RawB {
    static constexpr int TASKS = kUp * TcCfg<TERMS>::NOCT / TcCfg<TERMS>::NPROD;   // 2 (KC 64) or 1 (KC 32)
    static_assert(TASKS >= 1, "fewer producer tasks than threads");
    uint4 v[TASKS][kCyl];
};

// Lane bits 0-2 pick the time row within a group of 8, the next bits the
// octet, the rest (with the warp and the task index) the group: one warp load
// instruction then reads whole 32-byte sectors (all octets of 8 rows), and each
// quarter warp stores 8 distinct 16-byte rows of a core matrix (no conflicts).
template <int TERMS>
__device__ __forceinline__ void task_of(int tid, int i, int& t, int& oct) {
    using C = TcCfg<TERMS>;
    constexpr int RPW = 32 / C::NOCT;                 // time rows per warp and task (8 or 16)
    const int lane = tid & 31, warp = tid >> 5;
    oct = (lane >> 3) % C::NOCT;
    t = (lane & 7) + 8 * (lane / (8 * C::NOCT)) + RPW * warp + i * (C::NPROD / C::NOCT);
}

template <int TERMS>
__device__ __forceinline__ void load_b(const Seg& sg, long long row0, int kc, int tid, RawB<TERMS>& r) {
    using C = TcCfg<TERMS>;
#pragma unroll
    for (int i = 0; i < RawB<TERMS>::TASKS; ++i) {
        int t, oct;
        task_of<TERMS>(tid, i, t, oct);
        const int n0 = (C::KC / 2) * kc + 8 * oct;
        const uint8_t* rp = frame_row(sg, row0 + t) + 2 * n0;
#pragma unroll
        for (int c = 0; c < kCyl; ++c) r.v[i][c] = __ldg(reinterpret_cast<const uint4*>(rp + c * (kFeed * kPol)));
    }
}

// Build the B chunk: unpack, E-W toward beam j, split into FP16 hi (+ lo), and
// store row t = (yr, yi) per feed and row 128 + t = (yi, -yr).
template <int TERMS>
__device__ __forceinline__ void build_b(const RawB<TERMS>& r, uint32_t sel, const EwW& w, unsigned char* bhi,
                                        unsigned char* blo, int tid) {
    using C = TcCfg<TERMS>;
#pragma unroll
    for (int i = 0; i < RawB<TERMS>::TASKS; ++i) {
        int t, oct;
        task_of<TERMS>(tid, i, t, oct);
#pragma unroll
        for (int half = 0; half < 2; ++half) {           // feeds 4 half .. 4 half + 3 of the octet
            cp y0, y1;                                    // SoA: (n, n + 2) and (n + 1, n + 3)
#pragma unroll
            for (int c = 0; c < kCyl; ++c) {
                const uint32_t w0 = half ? r.v[i][c].z : r.v[i][c].x, w1 = half ? r.v[i][c].w : r.v[i][c].y;
                const uint32_t g0 = __byte_perm(w0, 0u, sel), g1 = __byte_perm(w1, 0u, sel);
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
            __half2 hr[4];
            uint32_t vre[4], vim[4];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                hr[f] = __floats2half2_rn(yr[f], yi[f]);
                vre[f] = h2u(hr[f]);
                vim[f] = h2u(__floats2half2_rn(yi[f], -yr[f]));
            }
            const int kg = 2 * oct + half;
            const int off_re = core_off<C::SBO>(t, kg), off_im = core_off<C::SBO>(128 + t, kg);
            *reinterpret_cast<uint4*>(bhi + off_re) = make_uint4(vre[0], vre[1], vre[2], vre[3]);
            *reinterpret_cast<uint4*>(bhi + off_im) = make_uint4(vim[0], vim[1], vim[2], vim[3]);
            if constexpr (C::B_LO) {
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    const float2 back = __half22float2(hr[f]);
                    const float lr = yr[f] - back.x, li = yi[f] - back.y;
                    vre[f] = h2u(__floats2half2_rn(lr, li));
                    vim[f] = h2u(__floats2half2_rn(li, -lr));
                }
                *reinterpret_cast<uint4*>(blo + off_re) = make_uint4(vre[0], vre[1], vre[2], vre[3]);
                *reinterpret_cast<uint4*>(blo + off_im) = make_uint4(vim[0], vim[1], vim[2], vim[3]);
            }
        }
    }
}

// One-thread bulk copy (TMA engine) of `bytes` into shared memory, completing
// on an mbarrier that expects that many bytes.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes) : "memory");
}


// MODE: 0 = detect and integrate, 1 = dump up-channelised voltages,
//       2 = dump the N-S/E-W beams of the GEMM (stage dump), 3 = stall check
//       (the MMA warp stays idle; the producers' bounded waits must run out).
//
// Warps 0-7 produce B chunks and run the up-channel passes out of TMEM; warp 8
// streams the twiddle chunks (bulk copies, NA-deep ring) and issues the MMAs.
// Chunks are numbered globally per CTA (item, pass, kc) so every barrier
// phase is consumed exactly once in order.
template <int TERMS, int MODE>
__global__ void __launch_bounds__(TcCfg<TERMS>::NT, 1) fused_tc_kernel(const __grid_constant__ Batch bt) {
    using C = TcCfg<TERMS>;
    constexpr int NA = C::NA;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;
    unsigned char* a_ring = smem;                                  // NA x A_STAGE
    unsigned char* b_ring = smem + NA * C::A_STAGE;                // 2 x B_STAGE
    float4* tw_s = reinterpret_cast<float4*>(b_ring + 2 * C::B_STAGE);
    uint64_t* mbar_s = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(tw_s) + 8 * 8 * 16);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool producer = warp < 8;
    const int ell = 32 * (warp & 3) + lane;           // TMEM lane (quarter = warp & 3)
    const int hh = (warp >> 2) & 1;                    // bin half: m = ell + 128 hh
    const int m = ell + 128 * hh;
    const uint32_t smem0 = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    const uint32_t bar0 = static_cast<uint32_t>(__cvta_generic_to_shared(&mbar_s[0]));
    // barriers: bfull[2] (8 producer warps), bempty[2] (MMA commit), afull[NA] (bulk copy),
    //           aempty[NA] (MMA commit), accfull (pass's last commit), tfree (8 producer warps)
    auto bfull = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto bempty = [&](int s) { return bar0 + 8u * (uint32_t)(2 + s); };
    auto afull = [&](int a) { return bar0 + 8u * (uint32_t)(4 + a); };
    auto aempty = [&](int a) { return bar0 + 8u * (uint32_t)(4 + NA + a); };
    const uint32_t accfull = bar0 + 8u * (uint32_t)(4 + 2 * NA);
    const uint32_t tfree = accfull + 8u;

    if (warp == 0) {
        const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(&tmem_base_s));
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(dst) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" :: "r"(bfull(i)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bempty(i)) : "memory");
        }
        for (int i = 0; i < NA; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(afull(i)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(aempty(i)) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(accfull) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" :: "r"(tfree) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
    }
    for (int i = tid; i < 64; i += C::NT) {
        const int it = i >> 3, c = i & 7;
        const float2 w0 = bt.tw128[(2 * it * c) & (kUp - 1)];
        const float2 w1 = bt.tw128[((2 * it + 1) * c) & (kUp - 1)];
        tw_s[i] = make_float4(w0.x, w1.x, w0.y, w1.y);
    }
    cta_sync();
    const uint32_t tmem = tmem_base_s;
    constexpr int PASSES = kTds * kPol;
    const unsigned long long wlim = bt.wait_ns ? bt.wait_ns : kWaitNs;
    // Tail items are split for the 1- and 3-term forms; the 2-term form, whose builders are
    // the most register- and L1-bound, measured slower with the extra epilogue.
    constexpr bool SPLIT = MODE == 0 && TERMS != 2;
    const Units units = make_units(bt.n_items, (int)gridDim.x, SPLIT);
    // this CTA's units are blockIdx.x + k gridDim.x: whole items first, then at most one half
    auto my_count = [&](int n) { return n > (int)blockIdx.x ? (n - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0; };
    const int n_my_whole = my_count(units.n_full), n_my_units = my_count(units.n_units);

    if (!producer) {
        // ------------------------------ MMA / copy warp ------------------------------
        // (MODE 3, the stall check: this warp stays idle, so no chunk is ever consumed)
        if (lane == 0 && MODE != 3) {
            uint32_t p_bfull = 0, p_afull = 0, p_aempty = 0, p_tfree = 0;
            long long c = 0;                                  // global chunk number
            long long c_copy = 0;                             // next twiddle chunk to copy
            const long long whole_chunks = (long long)n_my_whole * PASSES * C::NCH;
            const long long total = whole_chunks + (long long)(n_my_units - n_my_whole) * (PASSES / 2) * C::NCH;
            // twiddle image of the item that chunk cc belongs to; items only move forward,
            // so the segment search resumes where the previous lookup stopped
            int seg_cursor = 0;
            auto image_of = [&](long long cc) {
                const int k = cc < whole_chunks
                                  ? (int)(cc / (PASSES * C::NCH))
                                  : n_my_whole + (int)((cc - whole_chunks) / ((PASSES / 2) * C::NCH));
                int it, ps0, ps1, half;
                unit_of(units, (int)blockIdx.x + k * (int)gridDim.x, it, ps0, ps1, half);
                while (seg_cursor + 1 < bt.n_segs && bt.segs[seg_cursor + 1].item_begin <= it) ++seg_cursor;
                return bt.segs[seg_cursor].a_img;
            };
            auto issue_copy = [&](long long cc) {
                const int a = (int)(cc % NA), kc = (int)(cc % C::NCH);
                const unsigned char* a_hi = image_of(cc);
                unsigned char* st = a_ring + a * C::A_STAGE;
                mbar_expect(afull(a), C::A_STAGE);
                bulk_g2s(smem0 + (uint32_t)(st - smem), a_hi + (size_t)kc * C::OPER, C::OPER, afull(a));
                if constexpr (C::A_LO)
                    bulk_g2s(smem0 + (uint32_t)(st + C::OPER - smem), a_hi + (size_t)(C::NCH + kc) * C::OPER,
                             C::OPER, afull(a));
            };
            bool ok = true;
            // prologue: the first NA - 1 twiddle chunks
            for (; c_copy < total && c_copy < NA - 1; ++c_copy) issue_copy(c_copy);
            for (; c < total && ok; ++c) {
                const int s = (int)(c & 1), a = (int)(c % NA), kc = (int)(c % C::NCH);
                if (kc == 0 && c > 0) {
                    // the previous pass's accumulator has been read by the producers
                    if (!mbar_wait(tfree, p_tfree, wlim)) ok = false;
                    p_tfree ^= 1u;
                }
                if (!mbar_wait(bfull(s), (p_bfull >> s) & 1u, wlim)) ok = false;
                p_bfull ^= 1u << s;
                if (!mbar_wait(afull(a), (p_afull >> a) & 1u, wlim)) ok = false;
                p_afull ^= 1u << a;
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ahi = smem0 + (uint32_t)(a_ring + a * C::A_STAGE - smem), alo = ahi + C::OPER;
                const uint32_t bhi = smem0 + (uint32_t)(b_ring + s * C::B_STAGE - smem), blo = bhi + C::OPER;
#pragma unroll
                for (int ks = 0; ks < C::KC / 16; ++ks) {
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        const uint32_t d = tmem + mt * 256;
                        const uint32_t aoff = mt * 16 * C::SBO + ks * 256;
                        const uint64_t da = smem_desc(ahi + aoff, 128, C::SBO);
                        const uint64_t db = smem_desc(bhi + ks * 256, 128, C::SBO);
                        mma_f16(d, da, db, (kc | ks) ? 1u : 0u);
                        if constexpr (C::B_LO) mma_f16(d, da, smem_desc(blo + ks * 256, 128, C::SBO), 1u);
                        if constexpr (C::A_LO) mma_f16(d, smem_desc(alo + aoff, 128, C::SBO), db, 1u);
                    }
                }
                mma_commit(bempty(s));
                mma_commit(aempty(a));
                if (kc == C::NCH - 1) mma_commit(accfull);
                // refill: chunk c + NA - 1 goes into the stage of chunk c - 1 once its MMAs are done
                if (c_copy < total) {
                    if (c_copy >= NA) {
                        const int ra = (int)(c_copy % NA);
                        if (!mbar_wait(aempty(ra), (p_aempty >> ra) & 1u, wlim)) ok = false;
                        p_aempty ^= 1u << ra;
                    }
                    issue_copy(c_copy);
                    ++c_copy;
                }
                if (abort_s) ok = false;
            }
            if (!ok) abort_s = 1;
        }
        __syncwarp();
    } else {
        // ------------------------------ producer warps ------------------------------
        const uint32_t tlane = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + hh * 256;
        uint32_t p_bempty = 0, p_acc = 0;
        long long c = 0;
        bool ok = true;
        for (int k = 0; k < n_my_units && ok; ++k) {
            int item, ps0, ps1, half;
            unit_of(units, (int)blockIdx.x + k * (int)gridDim.x, item, ps0, ps1, half);
            int sgi = 0;
            while (sgi + 1 < bt.n_segs && bt.segs[sgi + 1].item_begin <= item) ++sgi;
            const Seg& sg = bt.segs[sgi];
            const int local = item - sg.item_begin;
            const int F = local >> 2, j = local & 3;
            EwW w;
            load_ew_frame(sg, bt.ew, F, j, w);
            float2 acc[kSub];
#pragma unroll
            for (int q = 0; q < kSub; ++q) acc[q] = make_float2(0.f, 0.f);
            RawB<TERMS> raw;
            load_b<TERMS>(sg, (long long)F * kFrame + (ps0 >> 1) * kUp, 0, tid, raw);
            for (int ps = ps0; ps < ps1 && ok; ++ps) {
                const int blk = ps >> 1, pol = ps & 1;
                const uint32_t sel = 0x4400u | ((2u + pol) << 4) | (uint32_t)pol;
                for (int kc = 0; kc < C::NCH && ok; ++kc, ++c) {
                    const int s = (int)(c & 1);
                    if (c >= 2) {
                        if (!mbar_wait(bempty(s), (p_bempty >> s) & 1u, wlim)) ok = false;
                        p_bempty ^= 1u << s;
                    }
                    unsigned char* sb_hi = b_ring + s * C::B_STAGE;
                    unsigned char* sb_lo = sb_hi + C::OPER;
                    RawB<TERMS> cur = raw;
                    const bool last = kc + 1 == C::NCH;
                    if (!last || ps + 1 < ps1) {
                        const int nblk = last ? ((ps + 1) >> 1) : blk;
                        load_b<TERMS>(sg, (long long)F * kFrame + nblk * kUp, last ? 0 : kc + 1, tid, raw);
                    }
                    build_b<TERMS>(cur, sel, w, sb_hi, sb_lo, tid);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bfull(s));
                    if (abort_s) ok = false;
                }
                if (!ok) break;
                if (!mbar_wait(accfull, p_acc, wlim)) ok = false;
                p_acc ^= 1u;
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if constexpr (MODE == 2) {
                    float2* d = bt.dump + ((((long long)(F * kTds + blk) * kPol + pol) * kEw + j) * kNs + m) * kUp;
                    for (int c4 = 0; c4 < 4; ++c4) {
                        float re[32], im[32];
                        tmem_ld32f(tlane + 32 * c4, re);
                        tmem_ld32f(tlane + 128 + 32 * c4, im);
                        for (int b = 0; b < 32; ++b) d[32 * c4 + b] = make_float2(re[b], im[b]);
                    }
                } else {
                    upchan_pass1_split(tlane, tw_s, 0, 1);
                    tmem_wait_st();
                    upchan_pass2_split(tlane, acc,
                                       MODE == 1 ? bt.dump + ((((long long)(F * kTds + blk) * kPol + pol) * kEw + j) * kNs + m) * kUp
                                                 : nullptr,
                                       0, 1);
                }
                // this warp's TMEM reads of the pass are done
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(tfree);
                if constexpr (SPLIT) {
                    if (half < 0 && ps == PASSES / 2 - 1) {
                        // whole item: H0 (passes 0-2) parks in this CTA's slot (coalesced)
                        // until H1 is done
                        float* pk = bt.park + (size_t)blockIdx.x * (kSub * kNs) + m;
#pragma unroll
                        for (int q = 0; q < kSub; ++q) {
                            pk[q * kNs] = acc[q].x + acc[q].y;
                            acc[q] = make_float2(0.f, 0.f);
                        }
                    }
                }
            }
            if constexpr (MODE == 0) {
                if (ok) {
                    // forms that split items: each output is H0 + H1 (H = the two fine channels
                    // of a pair added first), split or not; the 2-term form: the running sum
                    float h1[kSub];
#pragma unroll
                    for (int q = 0; q < kSub; ++q) h1[q] = acc[q].x + acc[q].y;
                    float* o = sg.out + (long long)(kNs * j + m) * sg.beam_stride + F;
                    if (!SPLIT) {
#pragma unroll
                        for (int q = 0; q < kSub; ++q) o[(long long)q * sg.sub_stride] = h1[q];
                    } else if (half < 0) {
                        const float* pk = bt.park + (size_t)blockIdx.x * (kSub * kNs) + m;
                        float h0[kSub];
#pragma unroll
                        for (int q = 0; q < kSub; ++q) h0[q] = pk[q * kNs];
#pragma unroll
                        for (int q = 0; q < kSub; ++q) o[(long long)q * sg.sub_stride] = h0[q] + h1[q];
                    } else {
                        const int slot = item - units.n_full;
                        float* mine = bt.part + ((size_t)slot * 2 + half) * (kSub * kNs) + m;
#pragma unroll
                        for (int q = 0; q < kSub; ++q) mine[q * kNs] = h1[q];
                        if (second_half(bt.part_tok + (size_t)slot * kNs + m, bt.epoch, half)) {
                            const float* other = bt.part + ((size_t)slot * 2 + (half ^ 1)) * (kSub * kNs) + m;
                            float h0[kSub];
#pragma unroll
                            for (int q = 0; q < kSub; ++q) h0[q] = __ldcg(other + q * kNs);
#pragma unroll
                            for (int q = 0; q < kSub; ++q) o[(long long)q * sg.sub_stride] = h0[q] + h1[q];
                        }
                    }
                }
            }
        }
        if (!ok) abort_s = 1;
    }

    cta_sync();
    if (abort_s && tid == 0 && bt.status) atomicExch(bt.status, 1);
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tmem) : "memory");
    }
}

template <int TERMS, int MODE>
cudaError_t launch_tc(const Batch& b, int grid, cudaStream_t s) {
    if (b.n_items <= 0) return cudaSuccess;
    // the detecting 1- and 3-term kernels park and split: they need the plan's buffers
    if (MODE == 0 && TERMS != 2 && (!b.part || !b.park || !b.part_tok || grid > 2 * kMaxSplit))
        return cudaErrorInvalidValue;
    const int smem = (int)TcCfg<TERMS>::SMEM;
    // shared-memory opt-in, once per device (the outcome is kept and returned on every launch)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    static std::once_flag once[kMaxDevices];
    static cudaError_t result[kMaxDevices];
    std::call_once(once[dev], [&] {
        result[dev] = cudaFuncSetAttribute(fused_tc_kernel<TERMS, MODE>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
    if (result[dev] != cudaSuccess) return result[dev];
    fused_tc_kernel<TERMS, MODE><<<grid, TcCfg<TERMS>::NT, smem, s>>>(b);
    return cudaGetLastError();
}

}  // namespace

size_t tc_a_bytes(int terms) {
    const size_t one = (size_t)kNs * 2 * kFeed * 2;              // 256 rows x 512 K x FP16
    return terms == 3 ? 2 * one : one;
}

int tc_chunk_k(int terms) { return terms == 3 ? TcCfg<3>::KC : terms == 2 ? TcCfg<2>::KC : TcCfg<1>::KC; }

cudaError_t fused_tc_launch(const Batch& b, int terms, int mode, int grid, cudaStream_t s) {
    switch (terms * 10 + mode) {
        case 10: return launch_tc<1, 0>(b, grid, s);
        case 11: return launch_tc<1, 1>(b, grid, s);
        case 12: return launch_tc<1, 2>(b, grid, s);
        case 13: return launch_tc<1, 3>(b, grid, s);
        case 20: return launch_tc<2, 0>(b, grid, s);
        case 21: return launch_tc<2, 1>(b, grid, s);
        case 22: return launch_tc<2, 2>(b, grid, s);
        case 30: return launch_tc<3, 0>(b, grid, s);
        case 31: return launch_tc<3, 1>(b, grid, s);
        case 32: return launch_tc<3, 2>(b, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace chimebf
