// Internal interface between the host runtime (runtime.cpp) and the CUDA
// kernels (fused_fp32.cu).  Not part of the public C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace chimebf {

// Geometry the kernels are built for (Sec. 1, Sec. 2, Sec. 3, Table 1).
constexpr int kCyl = 4;          // cylinders
constexpr int kFeed = 256;       // feeds per cylinder (N)
constexpr int kPol = 2;          // polarisations
constexpr int kBins = 512;       // zero-padded N-S FFT length (N P, P = 2)
constexpr int kNs = 256;         // N-S beams kept by the clamp
constexpr int kEw = 4;           // E-W beams
constexpr int kUp = 128;         // up-channelisation FFT length
constexpr int kFds = 8;          // fine channels per output sub-channel
constexpr int kTds = 3;          // 128-sample blocks per output frame
constexpr int kSub = kUp / kFds; // 16 sub-channels
constexpr int kFrame = kUp * kTds;   // 384 samples per frame
constexpr int kInput = kCyl * kFeed * kPol;   // 2048 bytes per time sample
constexpr int kBeams = kEw * kNs;    // 1024 intensity beams
constexpr int kInvLen = kBins + kNs;  // per table: first beam of each bin, next beam of each beam

// Segments per launch (kernel-parameter space holds the descriptors).
constexpr int kMaxSegs = 160;
// Items of one launch that the FP32 kernel may split in two (at most half its grid).
constexpr int kMaxSplit = 512;

// One (request, channel): a frame stream made of `carry_rows` leftover rows
// followed by the request's new rows.
struct Seg {
    const uint8_t* vin;      // row 0 of this channel's new samples [n][2048]
    const uint8_t* carry;    // leftover rows [carry_rows][2048] (may be null)
    float* out;              // &out[beam 0][sub 16*chan][frame 0] of the request
    long long beam_stride;   // elements between beams  (16 * n_chan * n_frames)
    int sub_stride;          // elements between sub-channels (n_frames)
    int carry_rows;          // 0..383
    int n_frames;            // frames of this segment
    int table;               // row of the per-frequency tables
    int item_begin;          // first work item; 4 items (E-W beams) per frame
    int pad_;
    const float2* ew_frames; // tracking E-W beams: [n_frames][4 ew][4 cyl] phases, or null (static)
    const unsigned char* a_img;  // tensor-core form: FP16 twiddle image(s) of this segment's table
};

struct Batch {
    int n_segs;
    int n_items;
    const int16_t* lut;      // [n_tables][256]   clamp table, Eq. (1)
    const int16_t* inv;      // [n_tables][kInvLen] 512-row form: first beam of each bin, then the
                             // next beam with the same bin (-1 ends a list)
    const int16_t* order;    // [n_tables][256]   FP32 form: beam taken by consumer slot (TMEM lane + 128 x half)
    const float2* ew;        // [n_tables][4 ew][4 cyl] E-W phases
    const float2* tw512;     // [512] exp(-2 pi i e / 512)
    const float2* tw128;     // [128] exp(-2 pi i e / 128)
    float2* dump;            // debug: up-channelised voltages instead of detection
    int* status;                 // set non-zero by a kernel whose bounded wait expired
    unsigned long long wait_ns;  // bound on each device-side wait (0: the default, 2 s)
    float* part;                 // halves of split items [grid / 2 + 1][2][16][256] (null: no split)
    unsigned long long* part_tok;    // [grid / 2 + 1][256] handshake tokens (2 x epoch + half)
    unsigned long long epoch;        // this launch's number within the plan (from 1)
    float* park;                 // tensor-core form: first half of each CTA's item [grid][16][256]
    Seg segs[kMaxSegs];
};

// Launches of the CUDA code; each returns the launch status.
cudaError_t fused_fp32_launch(const Batch& b, int grid, cudaStream_t s);
cudaError_t fused_fp32_dump_launch(const Batch& b, int grid, cudaStream_t s);
cudaError_t debug_beams_launch(const uint8_t* vin, long long n_samples, const int16_t* lut,
                               const float2* ew, const float2* tw512, float2* out, cudaStream_t s);
cudaError_t debug_unpack_launch(const uint8_t* in, float* out, long long n, cudaStream_t s);
int fused_fp32_max_grid(int device);   // CTAs that fit at once (1 per SM)

// Tensor-core form: `terms` = 1, 2 or 3 GEMM terms; mode 0 = detect,
// 1 = dump up-channelised voltages, 2 = dump the N-S/E-W beams of the GEMM,
// 3 = stall check (1 term only): the MMA warp stays idle, so the producers'
// bounded waits run out and the kernel reports through `status`.
cudaError_t fused_tc_launch(const Batch& b, int terms, int mode, int grid, cudaStream_t s);
// Tensor-core form, 1 term, detection: clusters of two CTAs (grid even, at most one
// CTA per SM), each CTA 128 of the 256 bins of every item; no item is split.
cudaError_t fused_tc_pair_launch(const Batch& b, int grid, cudaStream_t s);
// The 512-row form (all bins of the zero-padded transform, clamp at the output) on clusters
// of four CTAs; the grid is the clusters that fit at once.
cudaError_t fused_tc_dft512_launch(const Batch& b, cudaStream_t s);
// Stall check of the cluster kernel (cluster 2 or 4 CTAs, one cluster): the MMA thread stays
// idle, the other waits run out against b.wait_ns and the kernel reports through b.status.
cudaError_t fused_tc_pair_stall_launch(const Batch& b, int cluster, cudaStream_t s);
size_t tc_a_bytes(int terms);    // bytes of one table's twiddle image(s)
cudaError_t skymap_launch(const float* in, int n_beams, long long per_beam, float* map, cudaStream_t s);
cudaError_t dedisperse_launch(const float* in, const int* delays, int n_sub, long long nf, long long n_out,
                              float* out, cudaStream_t s);
// Allocation-free dedispersion: the device's static delay table (address
// looked up once per device; the caller has made `device` current).
constexpr int kDdStaticMaxSub = kSub * 4096;    // 4096 channels x 16 sub-channels
constexpr int kMaxDevices = 64;
cudaError_t dedisperse_static_table(int device, int** table);
cudaError_t rescale_u8_launch(const float* in, long long rows, long long nf, uint8_t* codes, float* stats,
                              cudaStream_t s);
int tc_chunk_k(int terms);       // K elements per shared-memory chunk
// FP32 FMA-pipe probe: 4 CTAs per SM (at most n_sink / 256) of 256 threads, each
// thread `iters` (rounded up to 4) x 16 FFMA2 (paired) or 32 scalar FMA; *flop = flops issued.
cudaError_t fma_probe_launch(bool paired, long long iters, float* sink, long long n_sink, int sms, double* flop,
                             cudaStream_t s);

}  // namespace chimebf
