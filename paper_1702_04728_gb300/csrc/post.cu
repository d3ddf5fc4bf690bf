// Kernels that run on the fan-beam output (arXiv 1702.04728, Sec. 3, Sec. 3.3,
// Table 1): the frequency- and time-summed sky map of Fig. 3 and the 8-bit
// rescaling of the intensity listed in Table 1.
#include "bf_internal.h"

#include <algorithm>
#include <cstdint>
#include <mutex>

namespace chimebf {
namespace {

constexpr int kMapThreads = 256;

// One CTA per beam: sum of the beam's [n_sub][n_frames] block (contiguous),
// fixed-order tree reduction in FP32.
__global__ void __launch_bounds__(kMapThreads) skymap_kernel(const float* __restrict__ in, long long per_beam,
                                                             float* __restrict__ map) {
    __shared__ float red[kMapThreads / 32];
    const float* p = in + (long long)blockIdx.x * per_beam;
    float s = 0.f;
    const long long n4 = per_beam / 4;
    const bool al = ((reinterpret_cast<uintptr_t>(p) & 15) == 0);
    if (al) {
        const float4* p4 = reinterpret_cast<const float4*>(p);
        for (long long i = threadIdx.x; i < n4; i += kMapThreads) {
            const float4 v = __ldg(p4 + i);
            s += (v.x + v.y) + (v.z + v.w);
        }
        for (long long i = 4 * n4 + threadIdx.x; i < per_beam; i += kMapThreads) s += __ldg(p + i);
    } else {
        for (long long i = threadIdx.x; i < per_beam; i += kMapThreads) s += __ldg(p + i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = threadIdx.x < kMapThreads / 32 ? red[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) map[blockIdx.x] = t;
    }
}

// One thread per (beam, sub-channel) row: mean and population standard
// deviation over the row's frames, then code = clip(floor(64 + 16 (x - mean) /
// std + 1/2), 0, 255), a constant row giving 64.  FP32: the sums run over x -
// x0 (x0 = the row's first frame), which keeps a constant row exactly constant
// (mean = x0, std = 0) and makes the rounding error of the mean scale with the
// row's spread instead of its level.  Valid for |x - mean| below ~1e18 (the
// squares stay finite).  A CTA stages its 32 rows through shared
// memory with coalesced loads; when the row length is a multiple of 4 (and the
// code array 4-byte aligned) the codes
// go back through shared memory as 32-bit words (rows padded by one word, no
// bank conflicts) and leave with coalesced stores, row by row.  Rows longer
// than the stage are read and written directly.
constexpr int kU8Rows = 32;
constexpr int kU8Stage = 256;          // frames staged per row
constexpr int kU8Words = kU8Stage / 4 + 1;

__global__ void __launch_bounds__(kU8Rows) rescale_u8_kernel(const float* __restrict__ in, long long rows,
                                                               long long nf, uint8_t* __restrict__ codes,
                                                               float* __restrict__ stats) {
    __shared__ float st[kU8Rows][kU8Stage + 1];
    __shared__ uint32_t cw[kU8Rows][kU8Words];
    const long long r0 = (long long)blockIdx.x * kU8Rows;
    const long long r = r0 + threadIdx.x;
    const bool staged = nf <= kU8Stage;
    const bool words = staged && (nf & 3) == 0 && (reinterpret_cast<uintptr_t>(codes) & 3) == 0;
    const int nr = (int)min((long long)kU8Rows, rows - r0);
    if (staged) {
        // the CTA's rows are contiguous: walk the block with 32 consecutive floats per load
        // instruction, many loads in flight (the row and column advance without a division)
        const float* src = in + r0 * nf;
        const long long n = (long long)nr * nf;
        int rr = (int)(threadIdx.x / nf);
        long long f = threadIdx.x - rr * nf;
        const long long step_r = kU8Rows / nf, step_f = kU8Rows % nf;
#pragma unroll 16
        for (long long i = threadIdx.x; i < n; i += kU8Rows) {
            st[rr][f] = __ldg(src + i);
            rr += (int)step_r;
            f += step_f;
            if (f >= nf) {
                f -= nf;
                ++rr;
            }
        }
        __syncthreads();
    }
    if (r < rows) {
        const float* x = in + r * nf;
        auto val = [&](long long f) -> float { return staged ? st[threadIdx.x][f] : __ldg(x + f); };
        const float x0 = val(0);
        float s = 0.f;
        for (long long f = 1; f < nf; ++f) s += val(f) - x0;
        const float mean = x0 + s / (float)nf;
        float q = 0.f;
        for (long long f = 0; f < nf; ++f) {
            const float d = val(f) - mean;
            q = fmaf(d, d, q);
        }
        const float sd = sqrtf(q / (float)nf);
        if (stats) {
            stats[2 * r] = mean;
            stats[2 * r + 1] = sd;
        }
        const float scale = sd > 0.f ? 16.f / sd : 0.f;
        auto code = [&](long long f) -> uint32_t {
            float v = 64.f;
            if (sd > 0.f) v = floorf(fmaf(val(f) - mean, scale, 64.5f));
            v = v < 0.f ? 0.f : (v > 255.f ? 255.f : v);
            return (uint32_t)v;
        };
        if (words) {
            for (int w = 0; w < (int)(nf >> 2); ++w)
                cw[threadIdx.x][w] = code(4 * w) | code(4 * w + 1) << 8 | code(4 * w + 2) << 16 |
                                     code(4 * w + 3) << 24;
        } else {
            uint8_t* c = codes + r * nf;
            for (long long f = 0; f < nf; ++f) c[f] = (uint8_t)code(f);
        }
    }
    if (words) {
        __syncthreads();
        // row r0 + rr starts at a 4-byte boundary of `codes` (nf is a multiple of 4)
        const int nw = (int)(nf >> 2);
        for (int rr = 0; rr < nr; ++rr) {
            uint32_t* dst = reinterpret_cast<uint32_t*>(codes + (r0 + rr) * nf);
            for (int w = threadIdx.x; w < nw; w += kU8Rows) dst[w] = cw[rr][w];
        }
    }
}

// Incoherent dedispersion to one DM: series[beam][t] = sum over sub-channels s
// (in order) of in[beam][s][t + d_s], t < n_out.  Threads run along t, so each
// sub-channel row is read with coalesced loads.
__global__ void dedisperse_kernel(const float* __restrict__ in, const int* __restrict__ delays, int n_sub,
                                  long long nf, long long n_out, float* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int beam = blockIdx.y;
    if (t >= n_out) return;
    const float* row = in + (long long)beam * n_sub * nf + t;
    float acc = 0.f;
    for (int s = 0; s < n_sub; ++s) acc += __ldg(row + (long long)s * nf + delays[s]);
    out[(long long)beam * n_out + t] = acc;
}

// Delay table of the allocation-free dedispersion entry point: one array per
// device, shared by every plan of the process (see bf_dedisperse_static).
__device__ __align__(256) int g_dd_delays[kDdStaticMaxSub];


// FP32 FMA-pipe probe: every thread runs kProbeChains independent chains of
// packed (FFMA2) or scalar FMAs, so the pipe, not latency, sets the rate.  The
// chains converge to c / (1 - b) and stay finite; their sum is stored so that
// no FMA can be removed.
constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 16;

template <bool kPair>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(long long iters, float* __restrict__ sink) {
    float2 a[kProbeChains];
    const float t = 1e-3f * (float)(threadIdx.x & 31);
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = make_float2(t + (float)k, t - (float)k);
    const float2 b = make_float2(0.9999f, 0.99991f), c = make_float2(1e-4f, 2e-4f);
#pragma unroll 1
    for (long long i = 0; i < iters; i += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int k = 0; k < kProbeChains; ++k) {
                if constexpr (kPair) {
                    a[k] = __ffma2_rn(a[k], b, c);
                } else {
                    a[k].x = __fmaf_rn(a[k].x, b.x, c.x);
                    a[k].y = __fmaf_rn(a[k].y, b.y, c.y);
                }
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += a[k].x + a[k].y;
    sink[(long long)blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace

cudaError_t dedisperse_static_table(int device, int** table) {
    static std::mutex mu;
    static int* ptrs[kMaxDevices] = {};
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!ptrs[device]) {
        // once per device, with that device current (the caller has set it)
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_dd_delays);
        if (e != cudaSuccess) return e;
        ptrs[device] = static_cast<int*>(p);
    }
    *table = ptrs[device];
    return cudaSuccess;
}

cudaError_t dedisperse_launch(const float* in, const int* delays, int n_sub, long long nf, long long n_out,
                              float* out, cudaStream_t s) {
    if (n_out <= 0) return cudaSuccess;
    dim3 grid((unsigned)((n_out + 127) / 128), kBeams);
    dedisperse_kernel<<<grid, 128, 0, s>>>(in, delays, n_sub, nf, n_out, out);
    return cudaGetLastError();
}

cudaError_t skymap_launch(const float* in, int n_beams, long long per_beam, float* map, cudaStream_t s) {
    if (n_beams <= 0) return cudaSuccess;
    skymap_kernel<<<n_beams, kMapThreads, 0, s>>>(in, per_beam, map);
    return cudaGetLastError();
}

cudaError_t fma_probe_launch(bool paired, long long iters, float* sink, long long n_sink, int sms, double* flop,
                             cudaStream_t s) {
    const long long blocks = std::min<long long>(4LL * sms, n_sink / kProbeThreads);
    if (blocks <= 0 || iters <= 0) return cudaErrorInvalidValue;
    const long long it4 = (iters + 3) / 4 * 4;
    *flop = (double)blocks * kProbeThreads * (double)it4 * kProbeChains * 4.0;
    if (paired)
        fma_probe_kernel<true><<<(unsigned)blocks, kProbeThreads, 0, s>>>(it4, sink);
    else
        fma_probe_kernel<false><<<(unsigned)blocks, kProbeThreads, 0, s>>>(it4, sink);
    return cudaGetLastError();
}

cudaError_t rescale_u8_launch(const float* in, long long rows, long long nf, uint8_t* codes, float* stats,
                              cudaStream_t s) {
    if (rows <= 0 || nf <= 0) return cudaSuccess;
    rescale_u8_kernel<<<(unsigned)((rows + kU8Rows - 1) / kU8Rows), kU8Rows, 0, s>>>(in, rows, nf, codes, stats);
    return cudaGetLastError();
}

}  // namespace chimebf
