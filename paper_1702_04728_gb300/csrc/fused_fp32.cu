// Fused FP32 fan-beam kernel for sm_103a (arXiv 1702.04728, Sec. 3).
//
// One CTA of 12 warps per SM owns a work item = (channel segment, output
// frame F, E-W beam j) and runs six passes over it, one per (128-sample
// block, polarisation).  Arithmetic is packed FP32x2 (FFMA2 / FADD2) in
// structure-of-arrays form: every value is a pair of two time samples (or two
// fine channels) that go through identical operations.
//
//  phase A, warps 0-7 (8 iterations per pass, 16 time samples each)
//    * warp w takes the row pair tau = 16 w + 2 it + {0, 1}, staged in shared
//      memory by cp.async, unpacks the 4+4-bit nibbles (Table 1) exactly and
//      forms E-W beam j (Sec. 3) -- applied before the N-S transform, legal
//      because both are linear and the phases do not depend on the feed;
//    * lanes 0-15 compute the even bins (FFT256 of y), lanes 16-31 the odd
//      bins (FFT256 of y exp(-i pi n / 256)) of the zero-padded 512-point N-S
//      FFT (Sec. 3.1), each as 16 x 16 with one shared-memory transpose; all
//      512 bins of the row pair land in the warp's row of a bin buffer;
//  gather + first up-channel pass, warps 8-11 (thread = N-S beams m, m + 128)
//    * bin L(m) of the clamp table (Eq. 1) is picked from the 8 rows of each
//      time residue pair, an 8-point DFT runs in registers, and the twiddled
//      result is parked in tensor memory (TMEM);
//  second up-channel pass (after the 128 samples of the block)
//    * 16-point DFTs from TMEM complete the 128-point FFT (Sec. 3.2), then
//      |.|^2 is accumulated into the 16 fftshifted sub-channels (Sec. 3).
//
// The corner turn of the paper's second kernel (time-slowest to
// time-fastest) is the gather into TMEM lanes: one (beam j, pol, block) is
// 256 beams x 128 samples x 8 B = 256 KB = all of TMEM.  Only packed input
// and float output touch global memory.
#include "device_common.cuh"

#include <cstdint>
#include <mutex>

namespace chimebf {
namespace {

constexpr int kWarps = 8;                   // phase-A (producer) warps: warp w loads row pair a = w
constexpr int kCons = 4;                    // gather / up-channel (consumer) warps, one per TMEM lane quarter
constexpr int kThreads = 32 * (kWarps + kCons);

// named barriers: 0 = whole CTA; FULL of bin buffer b; consumers only.  The release of a
// bin buffer (EMPTY) is an mbarrier the consumer warps arrive on, so producer warps wait
// for the consumers without waiting for each other.
constexpr int kBarFull = 1, kBarCons = 3;

// Register split (setmaxnreg): the launch gives every warp kRegLaunch registers per
// thread; the producer warpgroups (warps 0-7) raise theirs to kRegProd and the
// consumer warpgroup (warps 8-11) lowers its to kRegCons, within the same total.
constexpr int kRegLaunch = 168, kRegProd = 176, kRegCons = 152;
static_assert(kWarps * kRegProd + kCons * kRegCons <= (kWarps + kCons) * kRegLaunch,
              "the register split must fit in the launch's register file share");

// shared memory (float4 = one SoA pair: re0, re1, im0, im1)
constexpr int kBinsF4 = kWarps * kBins;             // 8 row pairs x 512 bins (one of two buffers)
constexpr int kYscF4 = kFeed;                        // per warp: its row pair's 256 phased feed lines
constexpr int kTbF4 = 2 * kFeed;                     // per warp: 2 halves x 16 x 16 (inside its own bin row)
constexpr int kRawB = 2 * kInput;                    // per producer warp and buffer: its two raw rows
constexpr size_t kSmemBins = 2 * (size_t)kBinsF4 * 16;   // double-buffered across iterations
constexpr size_t kSmemYsc = (size_t)kWarps * kYscF4 * 16;
constexpr size_t kSmemRaw = (size_t)kWarps * kRawB;      // raw rows (cp.async), one iteration ahead
constexpr size_t kSmemLut = 2 * kNs * sizeof(int);   // bins and beams in gather order
constexpr size_t kSmemTw = 8 * 8 * 16;               // pair twiddles of the first up-channel pass
constexpr size_t kSmemPark = (size_t)kSub * kNs * sizeof(float);   // first half of the current item
constexpr size_t kSmemTotal = kSmemBins + kSmemYsc + kSmemRaw + kSmemLut + kSmemTw + kSmemPark;
static_assert(kTbF4 == kBins, "a warp's transpose scratch is exactly its bin row");

__device__ __forceinline__ uint32_t smem_sa(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 128-bit shared-memory access by 32-bit shared address.  The XOR swizzles
// below become one LOP3 with an immediate per access on top of a per-lane base.
__device__ __forceinline__ void sts_cp(uint32_t addr, cp a) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};"
                 :: "r"(addr), "f"(a.re.x), "f"(a.re.y), "f"(a.im.x), "f"(a.im.y) : "memory");
}
__device__ __forceinline__ cp lds_cp(uint32_t addr) {
    cp a;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(a.re.x), "=f"(a.re.y), "=f"(a.im.x), "=f"(a.im.y) : "r"(addr) : "memory");
    return a;
}

// Phase A for one warp and its row pair (two time rows as SoA pairs):
//   in0/in1   the two raw rows
//   sel       byte permutation selecting polarisation pol of two feeds
//   ysc       this warp's phased feed lines [16 n2][16 n1] (swizzled, 4 KB)
//   tb        this warp's transpose scratch [2 halves][16][16] (8 KB; may be the bin row)
//   row_bins  the row pair's 512 bins (8 KB)
// Lanes 0-15 compute the even bins (FFT256 of y), lanes 16-31 the odd bins
// (FFT256 of y exp(-i pi n / 256)) of the zero-padded 512-point N-S FFT, lane
// n2 = lane & 15 in each half; `pt` holds that lane's twiddles.  Only warp-level
// synchronisation: no other warp touches this warp's scratch.
// Hooks: `after_ew` runs once in0/in1 have been consumed, `before_tb` before
// the transpose scratch is first written, `after_tb` after the transposed
// values are loaded (a slot for work that overlaps the last DFT).
template <class AfterEw, class BeforeTb, class AfterTb>
__device__ __forceinline__ void phase_a(const uint4 (&in0)[kCyl], const uint4 (&in1)[kCyl], uint32_t sel,
                                        const EwW& w, const PostTw& pt, uint32_t ysc, uint32_t tb, uint32_t row_bins,
                                        int lane, AfterEw after_ew, BeforeTb before_tb, AfterTb after_tb) {
    // unpack + E-W: lane holds feeds 8 lane .. 8 lane + 7 of both rows.  Feed n = 8 lane + 2k (+1)
    // sits at n2 = n & 15 = 8 (lane & 1) + 2k (+1), n1 = n >> 4 = lane >> 1; ysw(n2, n1) =
    // 16 n2 + (n1 ^ (n2 & 7) ^ 4 (n2 >> 3)) = 16 n2 + (((lane >> 1) ^ 4 (lane & 1)) ^ (n2 & 7)).
    const uint32_t yw = ysc + 16u * (uint32_t)(16 * 8 * (lane & 1) + (((lane >> 1) ^ (4 * (lane & 1)))));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        cp yA, yB;
#pragma unroll
        for (int c = 0; c < kCyl; ++c) {
            const uint32_t g0 = __byte_perm(word_of(in0[c], k), 0u, sel);
            const uint32_t g1 = __byte_perm(word_of(in1[c], k), 0u, sel);
            const float2 xiA = nib2<0>(g0, g1), xrA = nib2<1>(g0, g1);
            const float2 xiB = nib2<2>(g0, g1), xrB = nib2<3>(g0, g1);
            if (c == 0) {
                yA = {xrA, xiA};
                yB = {xrB, xiB};
            } else {
                yA.re = fma2(xiA, w.NI[c - 1], fma2(xrA, w.R[c - 1], yA.re));
                yA.im = fma2(xrA, w.I[c - 1], fma2(xiA, w.R[c - 1], yA.im));
                yB.re = fma2(xiB, w.NI[c - 1], fma2(xrB, w.R[c - 1], yB.re));
                yB.im = fma2(xrB, w.I[c - 1], fma2(xiB, w.R[c - 1], yB.im));
            }
        }
        // rows n2 = 2k and 2k + 1 of this lane's half: + 256 n2 bytes, low slot bits ^ n2
        sts_cp((yw ^ (uint32_t)(16 * (2 * k))) + 256u * (2 * k), yA);
        sts_cp((yw ^ (uint32_t)(16 * (2 * k + 1))) + 256u * (2 * k + 1), yB);
    }
    after_ew();
    __syncwarp();

    // half h = lane >> 4 of the padded FFT, lane handles n2 (both halves read the same lines):
    // ysw(n2, n1) = 16 n2 + (n1 ^ f), f = (n2 & 7) ^ 4 (n2 >> 3)
    const int h = lane >> 4, n2 = lane & 15;
    const uint32_t yr = ysc + 16u * (uint32_t)(16 * n2 + ((n2 & 7) ^ (4 * (n2 >> 3))));
    // loads in the order the first radix-4 stage of dft16 consumes them
    cp v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int n1 = 4 * (q & 3) + (q >> 2);
        v[n1] = lds_cp(yr ^ (uint32_t)(16 * n1));
    }
    if (h) {
        // odd bins: input times exp(-i pi n / 256) = exp(-2 pi i n1 / 32) * exp(-2 pi i n2 / 512);
        // the second factor is folded into the per-lane twiddles
#pragma unroll
        for (int n1 = 1; n1 < 16; ++n1) v[n1] = twiddle<32>(v[n1], n1);
    }
    dft16(v);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) v[k1] = cmulp(v[k1], pt.C[k1], pt.S[k1]);
    // the transpose scratch may share memory with bins still being read elsewhere
    before_tb();
    // transpose through tb (one 4 KB block per half): tsw(r, c) = 16 r + (c ^ (r & 7))
    const uint32_t tbl = tb + 16u * (uint32_t)(h * kFeed);
    {
        const uint32_t tw_ = tbl + 256u * (uint32_t)n2 + 16u * (uint32_t)(n2 & 7);
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) sts_cp(tw_ ^ (uint32_t)(16 * k1), v[k1]);
    }
    __syncwarp();
    const int k1 = n2;
    {
        const uint32_t tr_ = tbl + 16u * (uint32_t)k1;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int r = 4 * (q & 3) + (q >> 2);
            v[r] = lds_cp((tr_ ^ (uint32_t)(16 * (r & 7))) + 256u * r);
        }
    }
    after_tb();
    dft16(v);
    // every lane is done with the scratch before the bins (which may share its memory) are written
    __syncwarp();
    // bin of the 512-point padded FFT: L = 2 (k1 + 16 k2) + h = 32 k2 + (2 k1 + h), and
    // bsw(L) = 32 k2 + bsw(2 k1 + h) because bit 3 of L does not depend on k2
    const uint32_t row = row_bins + 16u * (uint32_t)bsw(2 * k1 + h);
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) sts_cp(row + 16u * 32u * k2, v[k2]);
}

// ---------------------------------------------------------------------------
// the fused kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bar_sync_n(int id, int n) { asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void bar_arrive_n(int id, int n) { asm volatile("bar.arrive %0, %1;" :: "r"(id), "r"(n) : "memory"); }

// 16-byte asynchronous global -> shared copy (no registers), grouped per iteration
__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

__device__ __forceinline__ uint4 lds_u4(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr)
                 : "memory");
    return v;
}

// Warps 0-7 (producers) run phase A for their row pairs; warps 8-11 (consumers,
// one per TMEM lane quarter) gather the clamped bins, run the first up-channel
// pass into TMEM and, after each block, the second pass and the detection for
// two bins each (m and m + 128).  The bin rows are double-buffered: producers
// arrive on the named barrier FULL[b] after writing buffer b, consumers arrive on
// the mbarrier EMPTY[b] after reading it, so phase A of iteration g + 1 overlaps
// the gather of iteration g and the second up-channel pass.  A producer can only
// be two iterations ahead of the slowest consumer and one FULL phase behind
// the others, so no barrier phase ever mixes iterations.  The EMPTY waits are
// bounded; on expiry the kernel carries on (keeping every barrier matched) and
// reports through the status word.
template <bool kDump>
__global__ void __launch_bounds__(kThreads, 1) fused_fp32_kernel(const __grid_constant__ Batch bt) {
    extern __shared__ __align__(256) unsigned char smem[];   // the swizzles XOR address bits 4-7
    float4* bins_all = reinterpret_cast<float4*>(smem);
    float4* ysc_all = reinterpret_cast<float4*>(smem + kSmemBins);
    unsigned char* raw_all = smem + kSmemBins + kSmemYsc;
    int* lut_s = reinterpret_cast<int*>(smem + kSmemBins + kSmemYsc + kSmemRaw);
    int* beam_s = lut_s + kNs;
    float4* tw_s = reinterpret_cast<float4*>(smem + kSmemBins + kSmemYsc + kSmemRaw + kSmemLut);
    float* park_s = reinterpret_cast<float*>(smem + kSmemBins + kSmemYsc + kSmemRaw + kSmemLut + kSmemTw);
    __shared__ uint32_t tmem_base_s;
    __shared__ __align__(8) uint64_t empty_s[2];
    __shared__ int expired_s;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int kAll = kThreads;
    const uint32_t empty0 = smem_sa(&empty_s[0]);

    if (warp == 0) {
        const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(&tmem_base_s));
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(dst) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // pair twiddles of the first up-channel pass: (b0, b1) = (2 it, 2 it + 1), c = 0..7
    for (int i = tid; i < 64; i += kThreads) {
        const int it = i >> 3, c = i & 7;
        const float2 w0 = bt.tw128[(2 * it * c) & (kUp - 1)];
        const float2 w1 = bt.tw128[((2 * it + 1) * c) & (kUp - 1)];
        tw_s[i] = make_float4(w0.x, w1.x, w0.y, w1.y);
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(empty0 + 8u * i), "n"(kCons) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        expired_s = 0;
    }
    cta_sync();
    const uint32_t tmem = tmem_base_s;
    constexpr int kPasses = kTds * kPol;
    const unsigned long long wlim = bt.wait_ns ? bt.wait_ns : kWaitNs;

    const Units units = make_units(bt.n_items, (int)gridDim.x, !kDump && bt.part != nullptr);
    static_assert(kTds * kPol == 6, "an item is two halves of three passes");

    if (warp < kWarps) {
        // ---------------------------------- producers ----------------------------------
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" :: "n"(kRegProd) : "memory");
        const uint32_t ysc_sa = smem_sa(ysc_all + warp * kYscF4);
        const uint32_t raw_sa = smem_sa(raw_all) + (uint32_t)(warp * kRawB) + 16u * lane;
        PostTw pt;
        load_post(bt.tw512, lane & 15, lane >> 4, pt);
        uint32_t g = 0;                                   // iterations done by this CTA
        for (int un = blockIdx.x; un < units.n_units; un += gridDim.x) {
            int item, ps0, ps1, half;
            unit_of(units, un, item, ps0, ps1, half);
            int sgi = 0;
            while (sgi + 1 < bt.n_segs && bt.segs[sgi + 1].item_begin <= item) ++sgi;
            const Seg& sg = bt.segs[sgi];
            const int local = item - sg.item_begin;
            const int F = local >> 2, j = local & 3;
            EwW w;
            load_ew_frame(sg, bt.ew, F, j, w);
            const long long row0 = (long long)F * kFrame + 16 * warp;
            // this warp's two rows of iteration (ps, it) into its raw buffer (own bytes only)
            auto fetch = [&](int ps, int it) {
                const long long r = row0 + (ps >> 1) * kUp + 2 * it;
                const uint8_t* p0 = frame_row(sg, r) + 16 * lane;
                const uint8_t* p1 = frame_row(sg, r + 1) + 16 * lane;
#pragma unroll
                for (int c = 0; c < kCyl; ++c) {
                    cp16(raw_sa + c * (kFeed * kPol), p0 + c * (kFeed * kPol));
                    cp16(raw_sa + kInput + c * (kFeed * kPol), p1 + c * (kFeed * kPol));
                }
                cp_commit();
            };
            auto load_raw = [&](uint4 (&r0)[kCyl], uint4 (&r1)[kCyl]) {
#pragma unroll
                for (int c = 0; c < kCyl; ++c) {
                    r0[c] = lds_u4(raw_sa + c * (kFeed * kPol));
                    r1[c] = lds_u4(raw_sa + kInput + c * (kFeed * kPol));
                }
            };
            // The current iteration's raw words are in registers.  Once the unpack has
            // consumed them, the next iteration's rows are copied into the raw buffer, and
            // they are read into registers during this iteration's last DFT.
            uint4 in0[kCyl], in1[kCyl];
            fetch(ps0, 0);
            cp_wait<0>();
            load_raw(in0, in1);
            for (int ps = ps0; ps < ps1; ++ps) {
                const int pol = ps & 1;
                const uint32_t sel = 0x4400u | ((2u + pol) << 4) | (uint32_t)pol;
                // two iterations per loop body give the scheduler room across the
                // iteration boundary (measured: unroll 1 / 2 / 4 = 1.652 / 1.632 / 1.652 ms)
#pragma unroll 2
                for (int it = 0; it < 8; ++it, ++g) {
                    const uint32_t b = g & 1u;
                    const bool more = it < 7 || ps + 1 < ps1;
                    const uint32_t row_bins = smem_sa(bins_all + b * kBinsF4 + warp * kBins);
                    phase_a(in0, in1, sel, w, pt, ysc_sa, row_bins, row_bins, lane,
                            [&] {
                                if (more) fetch(it < 7 ? ps : ps + 1, it < 7 ? it + 1 : 0);
                            },
                            [&] {
                                // buffer b is free once the consumers gathered it two iterations ago
                                // (release number g / 2 - 1 of buffer b)
                                if (g >= 2 && !mbar_wait(empty0 + 8u * b, ((g >> 1) + 1u) & 1u, wlim))
                                    expired_s = 1;
                            },
                            [&] {
                                // in0 / in1 were consumed by the unpack: the next rows replace them
                                if (more) {
                                    cp_wait<0>();
                                    load_raw(in0, in1);
                                }
                            });
                    bar_arrive_n(kBarFull + (int)b, kAll);
                }
            }
        }
    } else {
        // ---------------------------------- consumers ----------------------------------
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" :: "n"(kRegCons) : "memory");
        const int cq = warp - kWarps;                    // TMEM lane quarter
        const int ctid = tid - 32 * kWarps;
        const uint32_t tlane = tmem + (static_cast<uint32_t>(32 * cq) << 16);
        const int m0 = 32 * cq + lane;                   // consumer slots m0 (half 0) and m0 + 128 (half 1)
        uint32_t g = 0;
        for (int un = blockIdx.x; un < units.n_units; un += gridDim.x) {
            int item, ps0, ps1, half;
            unit_of(units, un, item, ps0, ps1, half);
            int sgi = 0;
            while (sgi + 1 < bt.n_segs && bt.segs[sgi + 1].item_begin <= item) ++sgi;
            const Seg& sg = bt.segs[sgi];
            const int local = item - sg.item_begin;
            const int F = local >> 2, j = local & 3;
            bar_sync_n(kBarCons, 32 * kCons);             // the previous item's table reads are done
            // consumer slot i (TMEM lane + 128 x half) takes beam order[i]
            for (int i = ctid; i < kNs; i += 32 * kCons) {
                const int bm = bt.order[sg.table * kNs + i];
                beam_s[i] = bm;
                lut_s[i] = bt.lut[sg.table * kNs + bm];
            }
            bar_sync_n(kBarCons, 32 * kCons);
            const int Lsw0 = bsw(lut_s[m0]), Lsw1 = bsw(lut_s[m0 + 128]);
            // the slots' beams (gather order); output addresses are formed where they are used
            auto out0 = [&] { return sg.out + (long long)(kNs * j + beam_s[m0]) * sg.beam_stride + F; };
            auto out1 = [&] { return sg.out + (long long)(kNs * j + beam_s[m0 + 128]) * sg.beam_stride + F; };
            float acc0[kSub], acc1[kSub];
#pragma unroll
            for (int s2 = 0; s2 < kSub; ++s2) {
                acc0[s2] = 0.f;
                acc1[s2] = 0.f;
            }
            for (int ps = ps0; ps < ps1; ++ps) {
                const int blk = ps >> 1, pol = ps & 1;
#pragma unroll 1
                for (int it = 0; it < 8; ++it, ++g) {
                    const uint32_t b = g & 1u;
                    bar_sync_n(kBarFull + (int)b, kAll);
                    const float4* bins = bins_all + b * kBinsF4;
                    // gather + 8-point DFT over a (tau = 16 a + b, b = 2 it, 2 it + 1), both bin halves
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const int Lsw = hh ? Lsw1 : Lsw0;
                        cp z[8];
#pragma unroll
                        for (int a = 0; a < 8; ++a) z[a] = ld_cp(bins + a * kBins + Lsw);
                        dft8(z);
                        const int b0 = 2 * it;
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            if (c) {
                                const float4 t = tw_s[it * 8 + c];
                                z[c] = cmulp(z[c], make_float2(t.x, t.y), make_float2(t.z, t.w));
                            }
                            tmem_st4(tlane + hh * 256 + 2 * (16 * c + b0), z[c].re.x, z[c].im.x, z[c].re.y,
                                     z[c].im.y);
                        }
                    }
                    __syncwarp();                                   // this warp's reads of buffer b are done
                    if (lane == 0) mbar_arrive(empty0 + 8u * b);
                }
                tmem_wait_st();
                // second pass: 16-point DFT over b for fine channels q = c + 8 d (this warp's lanes only)
                const long long dbase = ((((long long)(F * kTds + blk) * kPol + pol) * kEw + j) * kNs) * kUp;
                upchan_pass2(tlane, 0, acc0, kDump ? bt.dump + dbase + (long long)beam_s[m0] * kUp : nullptr);
                upchan_pass2(tlane, 1, acc1, kDump ? bt.dump + dbase + (long long)beam_s[m0 + 128] * kUp : nullptr);
                // the next pass's gathers overwrite these TMEM columns in this warp's program order
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if constexpr (!kDump) {
                    if (half < 0 && ps == kTds * kPol / 2 - 1) {
                        // whole item: H0 (passes 0-2) parks in shared memory until H1 is done
                        // (each thread reads back only its own words)
                        float* pk = park_s;
#pragma unroll
                        for (int s2 = 0; s2 < kSub; ++s2) {
                            pk[s2 * kNs + m0] = acc0[s2];
                            pk[s2 * kNs + m0 + 128] = acc1[s2];
                            acc0[s2] = 0.f;
                            acc1[s2] = 0.f;
                        }
                    }
                }
            }
            if constexpr (!kDump) {
                if (half < 0) {
                    // all loads before the first store: the stores could alias them as far as
                    // the compiler knows, and would otherwise serialise the loads
                    const float* pk = park_s;
                    float h[kSub];
#pragma unroll
                    for (int s2 = 0; s2 < kSub; ++s2) h[s2] = pk[s2 * kNs + m0];
                    float* o = out0();
#pragma unroll
                    for (int s2 = 0; s2 < kSub; ++s2) o[(long long)s2 * sg.sub_stride] = h[s2] + acc0[s2];
#pragma unroll
                    for (int s2 = 0; s2 < kSub; ++s2) h[s2] = pk[s2 * kNs + m0 + 128];
                    o = out1();
#pragma unroll
                    for (int s2 = 0; s2 < kSub; ++s2) o[(long long)s2 * sg.sub_stride] = h[s2] + acc1[s2];
                } else {
                    // half unit: publish this half; the second of the two halves to finish
                    // adds them (per thread: slots m0 and m0 + 128)
                    const int slot = item - units.n_full;
                    float* mine = bt.part + ((size_t)slot * 2 + half) * (kSub * kNs);
#pragma unroll
                    for (int s2 = 0; s2 < kSub; ++s2) {
                        mine[s2 * kNs + m0] = acc0[s2];
                        mine[s2 * kNs + m0 + 128] = acc1[s2];
                    }
                    if (second_half(bt.part_tok + (size_t)slot * kNs + m0, bt.epoch, half)) {
                        // H0 + H1 in either order: one addition of two terms is exact-commutative
                        const float* other = bt.part + ((size_t)slot * 2 + (half ^ 1)) * (kSub * kNs);
                        float h[kSub];
#pragma unroll
                        for (int s2 = 0; s2 < kSub; ++s2) h[s2] = __ldcg(other + s2 * kNs + m0);
                        float* o = out0();
#pragma unroll
                        for (int s2 = 0; s2 < kSub; ++s2) o[(long long)s2 * sg.sub_stride] = acc0[s2] + h[s2];
#pragma unroll
                        for (int s2 = 0; s2 < kSub; ++s2) h[s2] = __ldcg(other + s2 * kNs + m0 + 128);
                        o = out1();
#pragma unroll
                        for (int s2 = 0; s2 < kSub; ++s2) o[(long long)s2 * sg.sub_stride] = acc1[s2] + h[s2];
                    }
                }
            }
        }
    }

    cta_sync();
    if (expired_s && tid == 0 && bt.status) atomicExch(bt.status, 1);
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tmem) : "memory");
    }
}

// ---------------------------------------------------------------------------
// inspection kernels sharing the device code above
// ---------------------------------------------------------------------------

// Stages 1+2 of 4 consecutive rows per CTA (one warp pair), then the clamp gather.
__global__ void __launch_bounds__(64) debug_beams_kernel(const uint8_t* __restrict__ vin, long long T,
                                                          const int16_t* __restrict__ lut,
                                                          const float2* __restrict__ ew, const float2* __restrict__ tw512,
                                                          float2* __restrict__ out) {
    __shared__ __align__(256) float4 ysc[2 * kYscF4];     // 256-byte rows: the swizzles XOR address bits 4-7
    __shared__ __align__(256) float4 tbs[2][kTbF4];
    __shared__ __align__(256) float4 bins2[2 * kBins];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, e = warp;
    const long long t0 = (long long)blockIdx.x * 4;
    const int pol = blockIdx.y & 1, j = blockIdx.y >> 1;
    PostTw pt;
    load_post(tw512, lane & 15, lane >> 4, pt);
    EwW w;
    load_ew(ew, 0, j, w);
    uint4 in0[kCyl], in1[kCyl];
    const long long ra = min(t0 + 2 * e, T - 1), rb = min(t0 + 2 * e + 1, T - 1);
    load_row(vin + ra * kInput, lane, in0);
    load_row(vin + rb * kInput, lane, in1);
    const uint32_t sel = 0x4400u | ((2u + pol) << 4) | (uint32_t)pol;
    phase_a(in0, in1, sel, w, pt, smem_sa(ysc + e * kYscF4), smem_sa(tbs[warp]), smem_sa(bins2 + e * kBins), lane,
            [] {}, [] {}, [] {});
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * kNs; i += 64) {
        const int r = i >> 8, mm = i & 255;          // r: row 0..3 = slot (r >> 1), element (r & 1)
        const long long t = t0 + r;
        if (t >= T) continue;
        const float4 v = bins2[(r >> 1) * kBins + bsw(lut[mm])];
        out[((t * kPol + pol) * kEw + j) * kNs + mm] = (r & 1) ? make_float2(v.y, v.w) : make_float2(v.x, v.z);
    }
}

__global__ void debug_unpack_kernel(const uint8_t* __restrict__ in, float2* __restrict__ out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // byte i goes through the same path as a polarisation-0 byte of a feed A
    const uint32_t g = __byte_perm((uint32_t)in[i], 0u, 0x4420u);
    const float2 re = nib2<1>(g, g), im = nib2<0>(g, g);
    out[i] = make_float2(re.x, im.x);
}


// Shared-memory opt-in, and a check that the compiled kernel was given the
// registers per thread the setmaxnreg split assumes: with fewer, the producers'
// increase could not be granted, so such a build is refused instead of launched.
// Done once per device (the outcome is kept and returned on every launch); the flags
// have internal linkage, so two copies of the library in one process keep their own.
template <bool kDump>
cudaError_t prepare_fp32() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    static std::once_flag once[kMaxDevices];
    static cudaError_t result[kMaxDevices];
    std::call_once(once[dev], [&] {
        cudaFuncAttributes fa;
        cudaError_t r = cudaFuncGetAttributes(&fa, fused_fp32_kernel<kDump>);
        if (r == cudaSuccess && fa.numRegs < kRegLaunch) r = cudaErrorInvalidConfiguration;
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(fused_fp32_kernel<kDump>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kSmemTotal);
        result[dev] = r;
    });
    return result[dev];
}

}  // namespace

cudaError_t fused_fp32_launch(const Batch& b, int grid, cudaStream_t s) {
    if (b.n_items <= 0) return cudaSuccess;
    if (b.part && grid > 2 * kMaxSplit) return cudaErrorInvalidValue;
    cudaError_t e = prepare_fp32<false>();
    if (e != cudaSuccess) return e;
    fused_fp32_kernel<false><<<grid, kThreads, kSmemTotal, s>>>(b);
    return cudaGetLastError();
}

cudaError_t fused_fp32_dump_launch(const Batch& b, int grid, cudaStream_t s) {
    if (b.n_items <= 0) return cudaSuccess;
    cudaError_t e = prepare_fp32<true>();
    if (e != cudaSuccess) return e;
    fused_fp32_kernel<true><<<grid, kThreads, kSmemTotal, s>>>(b);
    return cudaGetLastError();
}

int fused_fp32_max_grid(int device) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    return sms;
}

cudaError_t debug_beams_launch(const uint8_t* vin, long long T, const int16_t* lut, const float2* ew,
                               const float2* tw512, float2* out, cudaStream_t s) {
    if (T == 0) return cudaSuccess;
    dim3 grid((unsigned)((T + 3) / 4), kPol * kEw);
    debug_beams_kernel<<<grid, 64, 0, s>>>(vin, T, lut, ew, tw512, out);
    return cudaGetLastError();
}

cudaError_t debug_unpack_launch(const uint8_t* in, float* out, long long n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    debug_unpack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, reinterpret_cast<float2*>(out), n);
    return cudaGetLastError();
}

}  // namespace chimebf
