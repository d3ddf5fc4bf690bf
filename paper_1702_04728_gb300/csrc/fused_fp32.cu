// Fused FP32 fan-beam kernel for sm_103a (arXiv 1702.04728, Sec. 3).
//
// One CTA (256 threads, one per SM) owns a work item = (channel segment,
// output frame F, E-W beam j) and runs six passes over it, one per
// (128-sample block, polarisation).  Arithmetic is packed FP32x2
// (FFMA2 / FADD2) in structure-of-arrays form: every value is a pair of two
// time samples (or two fine channels) that go through identical operations.
//
//  phase A (8 iterations per pass, 16 time samples each)
//    * warp w loads the row pair tau = 16 w + 2 it + {0, 1} with 128-bit loads,
//      unpacks the 4+4-bit nibbles (Table 1) exactly, and forms E-W beam j
//      (Sec. 3) -- applied before the N-S transform, legal because both are
//      linear and the phases do not depend on the feed;
//    * the warp pair (2q, 2q+1) shares the phased feed lines of its 4 rows; the
//      even warp computes the even bins (FFT256 of y), the odd warp the odd
//      bins (FFT256 of y exp(-i pi n / 256)) of the zero-padded 512-point
//      N-S FFT (Sec. 3.1), each as 16 x 16 with one shared-memory transpose;
//      all 512 bins of every row land in a shared-memory row;
//  gather + first up-channel pass (thread = N-S beam m)
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

namespace chimebf {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;       // 8: warp w loads row pair a = w
constexpr int kPairs = kWarps / 2;

// shared memory (float4 = one SoA pair: re0, re1, im0, im1)
constexpr int kBinsF4 = kWarps * kBins;             // 8 row pairs x 512 bins (one of two buffers)
constexpr int kYscF4 = 2 * kFeed;                    // per warp pair: 2 row pairs x 256 feeds
constexpr int kTbF4 = 2 * kFeed;                     // per warp: 2 row pairs x 16 x 16
constexpr size_t kSmemBins = 2 * (size_t)kBinsF4 * 16;   // double-buffered across iterations
constexpr size_t kSmemYsc = (size_t)kPairs * kYscF4 * 16;
constexpr size_t kSmemTb = (size_t)kWarps * kTbF4 * 16;
constexpr size_t kSmemLut = kNs * sizeof(int);
constexpr size_t kSmemTw = 8 * 8 * 16;               // pair twiddles of the first up-channel pass
constexpr size_t kSmemTotal = kSmemBins + kSmemYsc + kSmemTb + kSmemLut + kSmemTw;

// ---------------------------------------------------------------------------
// Phase A for one warp of a warp pair.
//   in0/in1  the two rows of this warp's row pair (slot e of the pair)
//   sel      byte permutation selecting polarisation pol of two feeds
//   ysc      the pair's phased feed lines [2 slots][16 n2][16 n1] (swizzled)
//   tb       this warp's transpose scratch [2 slots][16][16]
//   bins2    bins of the pair's row pair slot 0 (slot 1 at + kBins)
// e = warp & 1: the half of the padded FFT this warp computes, and the slot
// of the row pair it loads.
// ---------------------------------------------------------------------------
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

__device__ __forceinline__ void phase_a(const uint4 (&in0)[kCyl], const uint4 (&in1)[kCyl], uint32_t sel,
                                        const EwW& w, const PostTw& pt, uint32_t ysc, uint32_t tb, uint32_t bins2,
                                        int e, int lane, int bar_id) {
    // unpack + E-W: lane holds feeds 8 lane .. 8 lane + 7 of both rows.  Feed n = 8 lane + 2k (+1)
    // sits at n2 = n & 15 = 8 (lane & 1) + 2k (+1), n1 = n >> 4 = lane >> 1; ysw(n2, n1) =
    // 16 n2 + (n1 ^ (n2 & 7) ^ 4 (n2 >> 3)) = 16 n2 + (((lane >> 1) ^ 4 (lane & 1)) ^ (n2 & 7)).
    const uint32_t yw = ysc + 16u * (uint32_t)(e * kFeed + 16 * 8 * (lane & 1) + (((lane >> 1) ^ (4 * (lane & 1)))));
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
    pair_sync(bar_id);

    // lanes 0-15: row pair slot 0, lanes 16-31: slot 1; lane handles n2:
    // ysw(n2, n1) = 16 n2 + (n1 ^ f), f = (n2 & 7) ^ 4 (n2 >> 3)
    const int rp = lane >> 4, n2 = lane & 15;
    const uint32_t yr = ysc + 16u * (uint32_t)(rp * kFeed + 16 * n2 + ((n2 & 7) ^ (4 * (n2 >> 3))));
    cp v[16];
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) v[n1] = lds_cp(yr ^ (uint32_t)(16 * n1));
    if (e) {
        // odd bins: input times exp(-i pi n / 256) = exp(-2 pi i n1 / 32) * exp(-2 pi i n2 / 512);
        // the second factor is folded into the per-lane twiddles
#pragma unroll
        for (int n1 = 1; n1 < 16; ++n1) v[n1] = cmulp(v[n1], bc(cos32(n1)), bc(-sin32(n1)));
    }
    dft16(v);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) v[k1] = cmulp(v[k1], pt.C[k1], pt.S[k1]);
    // transpose through tb: tsw(r, c) = 16 r + (c ^ (r & 7))
    const uint32_t tbl = tb + 16u * (uint32_t)(rp * kFeed);
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
        for (int r = 0; r < 16; ++r) v[r] = lds_cp((tr_ ^ (uint32_t)(16 * (r & 7))) + 256u * r);
    }
    dft16(v);
    // bin of the 512-point padded FFT: L = 2 (k1 + 16 k2) + e = 32 k2 + (2 k1 + e), and
    // bsw(L) = 32 k2 + bsw(2 k1 + e) because bit 3 of L does not depend on k2
    const uint32_t row = bins2 + 16u * (uint32_t)(rp * kBins + bsw(2 * k1 + e));
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) sts_cp(row + 16u * 32u * k2, v[k2]);
}

// ---------------------------------------------------------------------------
// the fused kernel
// ---------------------------------------------------------------------------
template <bool kDump>
__global__ void __launch_bounds__(kThreads, 1) fused_fp32_kernel(const __grid_constant__ Batch bt) {
    extern __shared__ __align__(256) unsigned char smem[];   // the swizzles XOR address bits 4-7
    float4* bins_all = reinterpret_cast<float4*>(smem);
    float4* ysc_all = reinterpret_cast<float4*>(smem + kSmemBins);
    float4* tb_all = reinterpret_cast<float4*>(smem + kSmemBins + kSmemYsc);
    int* lut_s = reinterpret_cast<int*>(smem + kSmemBins + kSmemYsc + kSmemTb);
    float4* tw_s = reinterpret_cast<float4*>(smem + kSmemBins + kSmemYsc + kSmemTb + kSmemLut);
    __shared__ uint32_t tmem_base_s;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int e = warp & 1, q = warp >> 1;
    const uint32_t ysc_sa = smem_sa(ysc_all + q * kYscF4);
    const uint32_t tb_sa = smem_sa(tb_all + warp * kTbF4);


    // gather / second pass role: TMEM lane quarter = warp & 3, bin half = warp >> 2
    const int ell = 32 * (warp & 3) + lane;
    const int hh = warp >> 2;
    const int m = ell + 128 * hh;

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
    cta_sync();
    const uint32_t tmem = tmem_base_s;
    const uint32_t tlane = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16);

    PostTw pt;
    load_post(bt.tw512, lane & 15, e, pt);

    int par = 0;                     // bins buffer of the next iteration
    for (int item = blockIdx.x; item < bt.n_items; item += gridDim.x) {
        int sgi = 0;
        while (sgi + 1 < bt.n_segs && bt.segs[sgi + 1].item_begin <= item) ++sgi;
        const Seg& sg = bt.segs[sgi];
        const int local = item - sg.item_begin;
        const int F = local >> 2, j = local & 3;

        for (int i = tid; i < kNs; i += kThreads) lut_s[i] = bt.lut[sg.table * kNs + i];
        EwW w;
        load_ew_frame(sg, bt.ew, F, j, w);
        cta_sync();
        const int Lsw = bsw(lut_s[m]);

        float2 acc[kSub];
#pragma unroll
        for (int s = 0; s < kSub; ++s) acc[s] = make_float2(0.f, 0.f);

        const long long row0 = (long long)F * kFrame;
        // raw rows of the current iteration and the prefetched next one; the loop body is
        // unrolled twice with the roles swapped so the rows are never copied
        uint4 ra0[kCyl], ra1[kCyl], rb0[kCyl], rb1[kCyl];
        load_row(frame_row(sg, row0 + 16 * warp), lane, ra0);
        load_row(frame_row(sg, row0 + 16 * warp + 1), lane, ra1);

        for (int ps = 0; ps < kTds * kPol; ++ps) {
            const int blk = ps >> 1, pol = ps & 1;
            const uint32_t sel = 0x4400u | ((2u + pol) << 4) | (uint32_t)pol;
            auto step = [&](int it, const uint4 (&cur0)[kCyl], const uint4 (&cur1)[kCyl], uint4 (&nxt0)[kCyl],
                            uint4 (&nxt1)[kCyl]) {
                const bool more = it < 7 || ps + 1 < kTds * kPol;
                if (more) {
                    const int nit = it < 7 ? it + 1 : 0;
                    const int nblk = it < 7 ? blk : ((ps + 1) >> 1);
                    const long long r = row0 + nblk * kUp + 16 * warp + 2 * nit;
                    load_row(frame_row(sg, r), lane, nxt0);
                    load_row(frame_row(sg, r + 1), lane, nxt1);
                }
                // bins of this iteration: one buffer while the other is still being gathered
                float4* bins = bins_all + par * kBinsF4;
                par ^= 1;
                phase_a(cur0, cur1, sel, w, pt, ysc_sa, tb_sa, smem_sa(bins + (2 * q) * kBins), e, lane, 1 + q);
                cta_sync();
                // gather + 8-point DFT over a (tau = 16 a + b, b = 2 it, 2 it + 1)
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
                    tmem_st4(tlane + hh * 256 + 2 * (16 * c + b0), z[c].re.x, z[c].im.x, z[c].re.y, z[c].im.y);
                }
                // no barrier here: the next iteration writes the other bins buffer, and the
                // barrier after its phase A orders this gather before the buffer's reuse
            };
#pragma unroll 1
            for (int it = 0; it < 8; it += 2) {
                step(it, ra0, ra1, rb0, rb1);
                step(it + 1, rb0, rb1, ra0, ra1);
            }
            tmem_wait_st();
            cta_sync();
            // second pass: 16-point DFT over b for fine channels q = c + 8 d
            upchan_pass2(tlane, hh, acc,
                         kDump ? bt.dump + ((((long long)(F * kTds + blk) * kPol + pol) * kEw + j) * kNs + m) * kUp
                               : nullptr);
            // the next pass's first gather overwrites TMEM after two CTA barriers
        }

        if constexpr (!kDump) {
            float* o = sg.out + (long long)(kNs * j + m) * sg.beam_stride + F;
#pragma unroll
            for (int s = 0; s < kSub; ++s) o[(long long)s * sg.sub_stride] = acc[s].x + acc[s].y;
        }
        cta_sync();
    }

    cta_sync();
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
    __shared__ __align__(256) float4 ysc[kYscF4];         // 256-byte rows: the swizzles XOR address bits 4-7
    __shared__ __align__(256) float4 tbs[2][kTbF4];
    __shared__ __align__(256) float4 bins2[2 * kBins];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, e = warp;
    const long long t0 = (long long)blockIdx.x * 4;
    const int pol = blockIdx.y & 1, j = blockIdx.y >> 1;
    PostTw pt;
    load_post(tw512, lane & 15, e, pt);
    EwW w;
    load_ew(ew, 0, j, w);
    uint4 in0[kCyl], in1[kCyl];
    const long long ra = min(t0 + 2 * e, T - 1), rb = min(t0 + 2 * e + 1, T - 1);
    load_row(vin + ra * kInput, lane, in0);
    load_row(vin + rb * kInput, lane, in1);
    const uint32_t sel = 0x4400u | ((2u + pol) << 4) | (uint32_t)pol;
    phase_a(in0, in1, sel, w, pt, smem_sa(ysc), smem_sa(tbs[warp]), smem_sa(bins2), e, lane, 1);
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

}  // namespace

cudaError_t fused_fp32_launch(const Batch& b, int grid, cudaStream_t s) {
    if (b.n_items <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fused_fp32_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemTotal);
    if (e != cudaSuccess) return e;
    fused_fp32_kernel<false><<<grid, kThreads, kSmemTotal, s>>>(b);
    return cudaGetLastError();
}

cudaError_t fused_fp32_dump_launch(const Batch& b, int grid, cudaStream_t s) {
    if (b.n_items <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fused_fp32_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemTotal);
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
