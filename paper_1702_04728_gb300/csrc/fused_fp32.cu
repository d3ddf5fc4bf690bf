// Fused FP32 fan-beam kernel for sm_103a (arXiv 1702.04728, Sec. 3).
//
// One CTA (512 threads, one per SM) owns a work item = (channel segment,
// output frame F, E-W beam j) and runs six passes over it, one per
// (128-sample block, polarisation):
//
//  phase A (per iteration of 16 time samples, one warp per sample)
//    * 128-bit loads of the packed row, unpack of the 4+4-bit nibbles (Table 1);
//    * E-W phasing of the 4 cylinders toward beam j (Sec. 3) -- applied before
//      the N-S transform, which is legal because both are linear and the
//      phases do not depend on the feed;
//    * zero-padded 512-point N-S FFT of the 256 feeds (Sec. 3.1) as two
//      256-point FFTs (even and odd bins), each 16 x 16 in registers with one
//      shared-memory transpose; all 512 bins go to a shared-memory row;
//  gather + first up-channel pass (one thread per (N-S beam, time residue))
//    * the 256 bins of the clamp table (Eq. 1) are picked from the rows, an
//      8-point DFT over the 8 samples of one residue class runs in registers,
//      and the twiddled result is parked in tensor memory (TMEM, 256 KB);
//  second up-channel pass (after the 128 samples of the block)
//    * 16-point DFTs from TMEM complete the 128-point FFT (Sec. 3.2), then
//      |.|^2 is accumulated into the 16 fftshifted sub-channels (Sec. 3).
//
// The corner turn of the paper's second kernel (time-slowest to
// time-fastest) is the gather into TMEM lanes; nothing but packed input and
// float output touches global memory.
#include "bf_internal.h"

#include <cstdint>

namespace chimebf {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kScrStride = 17;                        // padded row (float2) of the per-warp scratch
constexpr int kScrWarp = 2 * 16 * kScrStride;         // float2 per warp: 32 rows of 17
constexpr int kBinsBuf = kWarps * kBins;              // float2 per bins buffer (16 rows of 512)

constexpr size_t kSmemBins = 2ull * kBinsBuf * sizeof(float2);          // 131072
constexpr size_t kSmemScr = (size_t)kWarps * kScrWarp * sizeof(float2); // 69632
constexpr size_t kSmemLut = kNs * sizeof(int);                          // 1024
constexpr size_t kSmemTw = kUp * sizeof(float2);                        // 1024
constexpr size_t kSmemTotal = kSmemBins + kSmemScr + kSmemLut + kSmemTw;

// ---------------------------------------------------------------------------
// complex helpers and small DFTs with compile-time twiddles
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 mul_neg_i(float2 a) { return make_float2(a.y, -a.x); }

// cos(2 pi e / 32) for e = 0..31, rounded from double precision.
__device__ __forceinline__ constexpr float cos32(int e) {
    constexpr float t[32] = {
        1.000000000e+00f, 9.807852804e-01f, 9.238795325e-01f, 8.314696123e-01f,
        7.071067812e-01f, 5.555702330e-01f, 3.826834324e-01f, 1.950903220e-01f,
        0.0f, -1.950903220e-01f, -3.826834324e-01f, -5.555702330e-01f,
        -7.071067812e-01f, -8.314696123e-01f, -9.238795325e-01f, -9.807852804e-01f,
        -1.000000000e+00f, -9.807852804e-01f, -9.238795325e-01f, -8.314696123e-01f,
        -7.071067812e-01f, -5.555702330e-01f, -3.826834324e-01f, -1.950903220e-01f,
        0.0f, 1.950903220e-01f, 3.826834324e-01f, 5.555702330e-01f,
        7.071067812e-01f, 8.314696123e-01f, 9.238795325e-01f, 9.807852804e-01f};
    return t[e & 31];
}
// sin(2 pi e / 32) = cos(2 pi (e - 8) / 32)
__device__ __forceinline__ constexpr float sin32(int e) { return cos32(e - 8); }

// a * exp(-2 pi i e / N) for N | 32 and a compile-time e (after unrolling).
template <int N>
__device__ __forceinline__ float2 twiddle(float2 a, int e) {
    constexpr float r = 7.071067812e-01f;
    const int k = (e * (32 / N)) & 31;               // angle in units of 2 pi / 32
    switch (k) {
        case 0: return a;
        case 4: return make_float2(r * (a.x + a.y), r * (a.y - a.x));
        case 8: return mul_neg_i(a);
        case 12: return make_float2(r * (a.y - a.x), -r * (a.x + a.y));
        case 16: return make_float2(-a.x, -a.y);
        case 20: return make_float2(-r * (a.x + a.y), r * (a.x - a.y));
        case 24: return make_float2(-a.y, a.x);
        case 28: return make_float2(r * (a.x - a.y), r * (a.x + a.y));
        default: return cmul(a, make_float2(cos32(k), -sin32(k)));
    }
}

// In-place forward DFT4 (exp(-i ...)), natural order.
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    const float2 s02 = a0 + a2, d02 = a0 - a2, s13 = a1 + a3, d13 = mul_neg_i(a1 - a3);
    a0 = s02 + s13;
    a2 = s02 - s13;
    a1 = d02 + d13;
    a3 = d02 - d13;
}

// In-place forward DFT8 (2 x 4): n = 2 n1 + n2, k = k1 + 4 k2.
__device__ __forceinline__ void dft8(float2 (&x)[8]) {
    dft4(x[0], x[2], x[4], x[6]);
    dft4(x[1], x[3], x[5], x[7]);
    x[3] = twiddle<8>(x[3], 1);
    x[5] = twiddle<8>(x[5], 2);
    x[7] = twiddle<8>(x[7], 3);
    float2 y[8];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        y[k1] = x[2 * k1] + x[2 * k1 + 1];
        y[k1 + 4] = x[2 * k1] - x[2 * k1 + 1];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = y[k];
}

// In-place forward DFT16 (4 x 4): n = 4 n1 + n2, k = k1 + 4 k2.
__device__ __forceinline__ void dft16(float2 (&x)[16]) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) x[4 * k1 + n2] = twiddle<16>(x[4 * k1 + n2], n2 * k1);
    float2 y[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 a0 = x[4 * k1], a1 = x[4 * k1 + 1], a2 = x[4 * k1 + 2], a3 = x[4 * k1 + 3];
        dft4(a0, a1, a2, a3);
        y[k1] = a0;
        y[k1 + 4] = a1;
        y[k1 + 8] = a2;
        y[k1 + 12] = a3;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = y[k];
}

// ---------------------------------------------------------------------------
// 4+4-bit unpack (Table 1): byte at position `pos` of `word`, high nibble real.
// The nibble is placed in the mantissa of 2^23 so the conversion is exact.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 unpack_byte(uint32_t word, int pos) {
    const uint32_t b = (word >> (8 * pos)) & 0xFFu;
    return make_float2(__uint_as_float(0x4B000000u | (b >> 4)) - 8388616.0f,
                       __uint_as_float(0x4B000000u | (b & 15u)) - 8388616.0f);
}

__device__ __forceinline__ uint32_t word_of(const uint4& v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// ---------------------------------------------------------------------------
// N-S + E-W for one time sample and polarisation, one warp.
//   in[c]  16 bytes of cylinder c: feeds 8*lane .. 8*lane+7, both pols
//   w[c]   E-W weight of cylinder c for the beam being formed
//   post   per-lane twiddles exp(-2 pi i n2 (2 k1 + h) / 512), k1 = 0..15
//   scr    this warp's scratch (kScrWarp float2)
//   row    512 float2 of shared memory: the zero-padded N-S bins, bin L at row[L]
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ns_ew_row(const uint4 (&in)[kCyl], int pol, const float2 (&w)[kCyl],
                                          const float2 (&post)[16], float2* scr, float2* row, int lane) {
    // E-W phasing on the unpacked voltages, written as y[n2][n1] with n = 16 n1 + n2.
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int pos = ((i & 1) << 1) | pol;
        float2 y = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < kCyl; ++c) {
            const float2 x = unpack_byte(word_of(in[c], i >> 1), pos);
            y.x += w[c].x * x.x - w[c].y * x.y;
            y.y += w[c].x * x.y + w[c].y * x.x;
        }
        scr[(((lane & 1) << 3) | i) * kScrStride + (lane >> 1)] = y;
    }
    __syncwarp();

    // Lanes 0-15 form the even bins (FFT256 of y), lanes 16-31 the odd bins
    // (FFT256 of y[n] exp(-i pi n / 256)).  Lane handles n2 = lane & 15.
    const int n2 = lane & 15, h = lane >> 4;
    float2 v[16];
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) v[n1] = scr[n2 * kScrStride + n1];
    // exp(-i pi n / 256) = exp(-2 pi i n1 / 32) exp(-2 pi i n2 / 512); the first
    // factor here, the second folded into post[].
#pragma unroll
    for (int n1 = 1; n1 < 16; ++n1) {
        const float cr = h ? cos32(n1) : 1.f;
        const float ci = h ? -sin32(n1) : 0.f;
        v[n1] = cmul(v[n1], make_float2(cr, ci));
    }
    dft16(v);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) v[k1] = cmul(v[k1], post[k1]);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) scr[((h << 4) | n2) * kScrStride + k1] = v[k1];
    __syncwarp();
    const int k1 = lane & 15;
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = scr[((h << 4) | j) * kScrStride + k1];
    dft16(v);
    // bin of the 512-point padded FFT: L = 2 (k1 + 16 k2) + h
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) row[2 * (k1 + 16 * k2) + h] = v[k2];
}

__device__ __forceinline__ void load_post(const float2* __restrict__ tw512, int lane, float2 (&post)[16]) {
    const int n2 = lane & 15, h = lane >> 4;
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) post[k1] = tw512[(n2 * (2 * k1 + h)) & (kBins - 1)];
}

__device__ __forceinline__ void load_row(const uint8_t* p, int lane, uint4 (&in)[kCyl]) {
#pragma unroll
    for (int c = 0; c < kCyl; ++c)
        in[c] = __ldg(reinterpret_cast<const uint4*>(p + c * (kFeed * kPol) + 16 * lane));
}

// ---------------------------------------------------------------------------
// tensor-memory access (tcgen05), one warp per 32-lane quarter
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tmem_st2(uint32_t taddr, float2 v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};"
                 :: "r"(taddr), "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float2 (&v)[16]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// CTA barrier that also orders tensor-memory accesses across it.
__device__ __forceinline__ void cta_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ const uint8_t* frame_row(const Seg& sg, long long row) {
    return row < sg.carry_rows ? sg.carry + row * kInput : sg.vin + (row - sg.carry_rows) * kInput;
}

// ---------------------------------------------------------------------------
// the fused kernel
// ---------------------------------------------------------------------------
template <bool kDump>
__global__ void __launch_bounds__(kThreads, 1) fused_fp32_kernel(const __grid_constant__ Batch bt) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2* bins = reinterpret_cast<float2*>(smem);
    float2* scr_all = reinterpret_cast<float2*>(smem + kSmemBins);
    int* lut_s = reinterpret_cast<int*>(smem + kSmemBins + kSmemScr);
    float2* tw128_s = reinterpret_cast<float2*>(smem + kSmemBins + kSmemScr + kSmemLut);
    __shared__ uint32_t tmem_base_s;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float2* scr = scr_all + warp * kScrWarp;

    // roles of the gather / second pass: TMEM lane quarter = warp & 3
    const int ell = 32 * (warp & 3) + lane;     // TMEM lane
    const int rsel = warp >> 2;                  // 0..3
    const int hh = rsel & 1;                     // N-S beam half: m = ell + 128 hh
    const int bsel = rsel >> 1;                  // gather: which of the two time residues
    const int chalf = rsel >> 1;                 // second pass: fine-channel half
    const int m = ell + 128 * hh;

    if (warp == 0) {
        const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(&tmem_base_s));
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(dst) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < kUp; i += kThreads) tw128_s[i] = bt.tw128[i];
    cta_sync();
    const uint32_t tmem = tmem_base_s;
    const uint32_t tlane = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16);

    float2 post[16];
    load_post(bt.tw512, lane, post);

    for (int item = blockIdx.x; item < bt.n_items; item += gridDim.x) {
        // locate the segment (descriptors are in kernel-parameter space)
        int sgi = 0;
        while (sgi + 1 < bt.n_segs && bt.segs[sgi + 1].item_begin <= item) ++sgi;
        const Seg& sg = bt.segs[sgi];
        const int local = item - sg.item_begin;
        const int F = local >> 2, j = local & 3;

        for (int i = tid; i < kNs; i += kThreads) lut_s[i] = bt.lut[sg.table * kNs + i];
        float2 w[kCyl];
#pragma unroll
        for (int c = 0; c < kCyl; ++c) w[c] = bt.ew[(sg.table * kEw + j) * kCyl + c];
        cta_sync();
        const int L = lut_s[m];

        float acc[kSub];
#pragma unroll
        for (int s = 0; s < kSub; ++s) acc[s] = 0.f;

        const long long row0 = (long long)F * kFrame;
        uint4 cur[kCyl];
        load_row(frame_row(sg, row0 + 16 * (warp & 7) + (warp >> 3)), lane, cur);

        for (int ps = 0; ps < kTds * kPol; ++ps) {
            const int blk = ps >> 1, pol = ps & 1;
            for (int it = 0; it < 8; ++it) {
                // prefetch the row this warp needs next
                uint4 nxt[kCyl];
                const int nit = it < 7 ? it + 1 : 0;
                const int nblk = it < 7 ? blk : ((ps + 1) >> 1);
                const bool more = it < 7 || ps + 1 < kTds * kPol;
                if (more) {
                    const long long r = row0 + nblk * kUp + 16 * (warp & 7) + 2 * nit + (warp >> 3);
                    load_row(frame_row(sg, r), lane, nxt);
                }
                // phase A: this warp's time sample tau = 16 (warp & 7) + 2 it + (warp >> 3)
                float2* rowbuf = bins + (it & 1) * kBinsBuf + warp * kBins;
                ns_ew_row(cur, pol, w, post, scr, rowbuf, lane);
                cta_sync();
                // gather + 8-point DFT over a (tau = 16 a + b), twiddle exp(-2 pi i b c / 128)
                {
                    const float2* bb = bins + (it & 1) * kBinsBuf + (8 * bsel) * kBins + L;
                    float2 z[8];
#pragma unroll
                    for (int a = 0; a < 8; ++a) z[a] = bb[a * kBins];
                    dft8(z);
                    const int b = 2 * it + bsel;
#pragma unroll
                    for (int c = 1; c < 8; ++c) z[c] = cmul(z[c], tw128_s[(b * c) & (kUp - 1)]);
#pragma unroll
                    for (int c = 0; c < 8; ++c) tmem_st2(tlane + hh * 256 + 32 * c + 2 * b, z[c]);
                }
                if (more) {
#pragma unroll
                    for (int c = 0; c < kCyl; ++c) cur[c] = nxt[c];
                }
            }
            tmem_wait_st();
            cta_sync();
            // second pass: 16-point DFT over b for fine channels q = c + 8 d
#pragma unroll 1
            for (int cc = 0; cc < 4; ++cc) {
                const int c = 4 * chalf + cc;
                float2 y[16];
                tmem_ld32(tlane + hh * 256 + 32 * c, y);
                dft16(y);
                if constexpr (kDump) {
                    float2* d = bt.dump + ((((long long)(F * kTds + blk) * kPol + pol) * kEw + j) * kNs + m) * kUp;
#pragma unroll
                    for (int dd = 0; dd < 16; ++dd) d[(c + 8 * dd + kUp / 2) & (kUp - 1)] = y[dd];
                } else {
#pragma unroll
                    for (int dd = 0; dd < 16; ++dd) acc[(dd + 8) & 15] += y[dd].x * y[dd].x + y[dd].y * y[dd].y;
                }
            }
            // the next pass's first gather overwrites TMEM: its barrier (after
            // phase A) orders it after these loads.
        }

        if constexpr (!kDump) {
            cta_sync();                                   // bins buffers free: reuse as combine area
            float* comb = reinterpret_cast<float*>(bins);
            if (chalf == 1) {
#pragma unroll
                for (int s = 0; s < kSub; ++s) comb[m * 17 + s] = acc[s];
            }
            cta_sync();
            if (chalf == 0) {
                float* o = sg.out + (long long)(kNs * j + m) * sg.beam_stride + F;
#pragma unroll
                for (int s = 0; s < kSub; ++s) o[(long long)s * sg.sub_stride] = acc[s] + comb[m * 17 + s];
            }
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
constexpr int kDbgWarps = 8;

__global__ void __launch_bounds__(kDbgWarps * 32) debug_beams_kernel(const uint8_t* __restrict__ vin, long long T,
                                                                     const int16_t* __restrict__ lut,
                                                                     const float2* __restrict__ ew,
                                                                     const float2* __restrict__ tw512,
                                                                     float2* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* scr = reinterpret_cast<float2*>(smem) + warp * (kScrWarp + kBins);
    float2* row = scr + kScrWarp;
    const long long task = (long long)blockIdx.x * kDbgWarps + warp;   // (t, pol, j)
    if (task >= T * kPol * kEw) return;
    const int j = task % kEw, pol = (task / kEw) % kPol;
    const long long t = task / (kEw * kPol);
    float2 post[16];
    load_post(tw512, lane, post);
    float2 w[kCyl];
#pragma unroll
    for (int c = 0; c < kCyl; ++c) w[c] = ew[j * kCyl + c];
    uint4 in[kCyl];
    load_row(vin + t * kInput, lane, in);
    ns_ew_row(in, pol, w, post, scr, row, lane);
    __syncwarp();
    float2* o = out + ((t * kPol + pol) * kEw + j) * kNs;
    for (int mm = lane; mm < kNs; mm += 32) o[mm] = row[lut[mm]];
}

__global__ void debug_unpack_kernel(const uint8_t* __restrict__ in, float2* __restrict__ out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t word = in[i];
    out[i] = unpack_byte(word, 0);
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
    const long long tasks = T * kPol * kEw;
    if (tasks == 0) return cudaSuccess;
    const size_t sm = (size_t)kDbgWarps * (kScrWarp + kBins) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(debug_beams_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    debug_beams_kernel<<<(unsigned)((tasks + kDbgWarps - 1) / kDbgWarps), kDbgWarps * 32, sm, s>>>(vin, T, lut, ew,
                                                                                                    tw512, out);
    return cudaGetLastError();
}

cudaError_t debug_unpack_launch(const uint8_t* in, float* out, long long n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    debug_unpack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, reinterpret_cast<float2*>(out), n);
    return cudaGetLastError();
}

}  // namespace chimebf
