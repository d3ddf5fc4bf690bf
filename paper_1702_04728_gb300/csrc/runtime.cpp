// Host runtime behind the C ABI of include/chimebf.h.
//
// A plan owns: FP64-derived device tables (clamp table of Eq. 1 and E-W
// phases per channel frequency, FFT twiddles), per-stream carry buffers (the
// < 384 samples left over between requests of one stream), and in SERVING
// mode a thread that batches queued requests of different streams into one
// launch of the fused kernel (continuous batching: requests that arrive while
// a batch runs join the next one, admitted against a memory budget).
#include "chimebf.h"
#include "bf_internal.h"

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <set>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

using namespace chimebf;

namespace {

constexpr double kC0 = 299792458.0;
constexpr double kPi = 3.14159265358979323846;
constexpr int kTableCap = 4096;        // default and largest number of per-frequency table slots
constexpr int kTcBlock = 64;           // tensor-core twiddle images are allocated 64 slots at a time
constexpr int kMaxInflight = 4;

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(BF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

struct StreamState {
    int n_chan = 0;
    std::vector<int> tables;        // per channel
    uint8_t* carry = nullptr;       // device [n_chan][kFrame - 1][2048]
    int carry_rows = 0;
    size_t carry_bytes = 0;
};

enum TicketState { T_QUEUED, T_INFLIGHT, T_DONE, T_ERROR };

struct Ticket {
    TicketState state = T_QUEUED;
    int64_t n_frames = 0;
    int err = 0;
    std::string msg;
    size_t bytes = 0;               // admission accounting
    uint64_t batch = 0;
    // timeline on the host's monotonic clock (seconds): submitted, its batch launched,
    // the batch's completion seen by the runtime
    double t_submit = 0, t_launch = 0, t_done = 0;
    double t_exec = 0;              // the batch's device time between its start and end events
};

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Job {
    uint64_t ticket;
    bf_request req;
    std::vector<double> freqs;
    int64_t track_frames = -1;      // >= 0: tracking E-W beams for this many output frames
    std::vector<float2> track;      // [n_chan][track_frames][4 ew][4 cyl] phases (FP64-derived)
};

// Pinned staging + device copy of one batch's tracking tables.
struct TrackBuf {
    size_t bytes = 0;
    float2* host = nullptr;
    float2* dev = nullptr;
};

struct InflightBatch {
    uint64_t id;
    cudaEvent_t ev;
    cudaEvent_t ev_start;                               // before the batch's first kernel (timing)
    std::vector<uint64_t> tickets;
    size_t bytes;
    std::vector<std::pair<size_t, uint8_t*>> release;   // carry buffers free once the batch is done
    TrackBuf track;                                     // tracking tables, back to the pool at retire
    std::vector<int> slots;                             // table slots the batch reads (one reference each)
};

}  // namespace

struct bf_plan_s {
    bf_config cfg{};
    std::vector<double> ns_sin, ew_sin;
    int device = 0;
    int grid = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    int16_t* d_lut = nullptr;
    int16_t* d_order = nullptr;               // FP32 form: gather order of the beams per table
    float2* d_ew = nullptr;
    float2* d_tw512 = nullptr;
    float2* d_tw128 = nullptr;
    // Per-frequency table slots (clamp table, gather order, E-W phases and, for the
    // tensor-core form, the FP16 twiddle image).  A slot is referenced by every open
    // stream that uses its frequency and by every unretired batch that reads it; a
    // new frequency takes a free slot, else the least recently used unreferenced one.
    std::map<uint64_t, int> table_of_freq;   // key: bit pattern of the double
    int table_cap = kTableCap;
    int n_slots = 0;                          // slots filled so far (< table_cap: a fresh one is free)
    std::vector<uint64_t> slot_key;
    std::vector<int> slot_refs;
    std::vector<uint64_t> slot_used;          // LRU clock of the slot's last lookup
    uint64_t lru_clock = 0;
    int terms = 0;                            // tensor-core GEMM terms (0: FP32 FFT form)
    bool dft512 = false;                      // BF_TC_DFT512: all 512 rows, the clamp at the output
    int16_t* d_inv = nullptr;                 // 512-row form: [table_cap][kInvLen] bin -> beams lists
    unsigned char* d_a512 = nullptr;          // 512-row form: the one FP16 image of the 512 x 512 DFT matrix
    std::vector<unsigned char*> atc_blocks;   // [kTcBlock][tc_a_bytes(terms)] FP16 twiddle images each
    int* h_status = nullptr;                  // mapped status word written by kernels
    int* d_delays = nullptr;                  // dedispersion delay table (grown on demand)
    size_t delays_cap = 0;
    int* d_status = nullptr;
    float* d_part = nullptr;                  // FP32 form: halves of split items (see Batch::part)
    unsigned long long* d_part_tok = nullptr;
    float* d_park = nullptr;                  // tensor-core form: per-CTA first halves (see Batch::park)
    unsigned long long launches = 0;          // launch epochs handed to the kernels

    std::mutex mu;
    std::condition_variable cv;
    std::unordered_map<uint64_t, StreamState> streams;
    std::unordered_map<uint64_t, Ticket> tickets;
    uint64_t next_ticket = 1;
    uint64_t next_batch = 1;
    std::deque<Job> queue;
    std::deque<InflightBatch> inflight;
    std::vector<cudaEvent_t> event_pool;
    std::multimap<size_t, uint8_t*> carry_pool;   // free carry buffers by size (reused, freed at destroy)
    std::multimap<size_t, TrackBuf> track_pool;   // free tracking-table buffers by size
    size_t mem_in_use = 0;      // bytes of requests in launched, unretired batches
    size_t queued_bytes = 0;    // bytes of requests waiting in the queue
    bool stop = false;
    std::thread worker;
};

namespace {

// Copy the N-S and E-W pointings of cfg (or the defaults) into p.
int fill_pointings(bf_plan_s* p, const bf_config* cfg) {
    for (int m = 0; m < kNs; ++m) {
        p->ns_sin[m] = cfg->ns_sin ? cfg->ns_sin[m] : (m - 127.5) / 128.0;
        if (!std::isfinite(p->ns_sin[m])) return fail(BF_EINVAL, "non-finite N-S pointing");
    }
    static const double deg[4] = {-0.6, -0.2, 0.2, 0.6};
    for (int j = 0; j < kEw; ++j) {
        p->ew_sin[j] = cfg->ew_sin ? cfg->ew_sin[j] : std::sin(deg[j] * kPi / 180.0);
        if (!std::isfinite(p->ew_sin[j])) return fail(BF_EINVAL, "non-finite E-W pointing");
    }
    return BF_OK;
}

// ---- tables -------------------------------------------------------------------

// Eq. (1): L = floor(N P f d sin(theta) / c + 0.5), product left to right in
// FP64, wrapped into [0, N P) (the wrap is the spatial aliasing of Sec. 3.3).
void clamp_table(const bf_plan_s* p, double f, int32_t* lut) {
    const double np = double(p->cfg.n_feed * p->cfg.pad);
    for (int m = 0; m < kNs; ++m) {
        const double arg = (((np * f) * p->cfg.feed_spacing_m) * p->ns_sin[m]) / kC0;
        long long L = (long long)std::floor(arg + 0.5);
        L %= kBins;
        if (L < 0) L += kBins;
        lut[m] = (int32_t)L;
    }
}

// E-W phasing (Sec. 3): cylinder c at c * D, beam j toward u_j:
// w[j][c] = exp(-2 pi i f c D u_j / c).
// E-W phases of the four beams (Sec. 3: exact phasing across the cylinders):
// w[j][c] = exp(-2 pi i frac(f c D u_j / c0)), products left to right in FP64.
void ew_phases(const bf_plan_s* p, double f, const double* u, float* ew) {
    for (int j = 0; j < kEw; ++j)
        for (int c = 0; c < kCyl; ++c) {
            const double cyc = (((f * c) * p->cfg.cyl_spacing_m) * u[j]) / kC0;
            const double fr = cyc - std::floor(cyc);
            ew[2 * (j * kCyl + c)] = (float)std::cos(-2.0 * kPi * fr);
            ew[2 * (j * kCyl + c) + 1] = (float)std::sin(-2.0 * kPi * fr);
        }
}

void ew_table(const bf_plan_s* p, double f, float* ew) { ew_phases(p, f, p->ew_sin.data(), ew); }

// Tracking buffer of at least `bytes` from the pool or new (pinned host + device).
int track_alloc(bf_plan_s* p, size_t bytes, TrackBuf* out) {
    auto it = p->track_pool.lower_bound(bytes);
    if (it != p->track_pool.end()) {
        *out = it->second;
        p->track_pool.erase(it);
        return BF_OK;
    }
    size_t cap = 4096;
    while (cap < bytes) cap <<= 1;
    TrackBuf t;
    t.bytes = cap;
    CK(cudaHostAlloc((void**)&t.host, cap, cudaHostAllocDefault));
    cudaError_t e = cudaMalloc((void**)&t.dev, cap);
    if (e != cudaSuccess) {
        cudaFreeHost(t.host);
        return cuda_fail(e, "cudaMalloc (tracking tables)");
    }
    *out = t;
    return BF_OK;
}

// Tensor-core twiddle image of `rows` rows: A[m][2n] = cos, A[m][2n+1] = sin
// of 2 pi n L(m) / 512 (the clamped rows of the zero-padded DFT, Eq. 1, with
// the clamp table as L; all 512 rows of the DFT matrix with L(m) = m), FP16
// hi (and lo = A - hi), laid out chunk by chunk exactly as the kernel's shared
// memory operand: 8-row x 16-byte core matrices, k-groups 128 B apart, row
// groups KC/8 * 128 B apart.
void tc_image(int terms, const int32_t* lut, int rows, std::vector<__half>& img) {
    const int KC = tc_chunk_k(terms);
    const size_t oper = (size_t)rows * KC;                // halves per chunk
    const size_t nch = 2 * kFeed / KC;
    const size_t one = oper * nch;
    img.assign(terms == 3 ? 2 * one : one, __float2half(0.f));
    for (int m = 0; m < rows; ++m)
        for (int n = 0; n < kFeed; ++n) {
            const long long e = ((long long)n * lut[m]) % kBins;
            const double th = 2.0 * kPi * (double)e / kBins;
            const double v[2] = {std::cos(th), std::sin(th)};
            for (int c = 0; c < 2; ++c) {
                const int kg = 2 * n + c;
                const size_t kc = kg / KC, k = kg % KC;
                const size_t off = kc * oper + ((size_t)(m >> 3) * (KC / 8) + (k >> 3)) * 64 + (m & 7) * 8 + (k & 7);
                const __half hi = __double2half(v[c]);
                img[off] = hi;
                if (terms == 3) img[one + off] = __double2half(v[c] - (double)__half2float(hi));
            }
        }
}

// The clamp (Eq. 1) read backwards for the 512-row form: inv[k] = the first beam m with
// L(m) = k and inv[512 + m] = the next beam after m with the same bin (-1 ends a list).
void inverse_clamp(const int32_t* lut, int16_t* inv) {
    for (int i = 0; i < kInvLen; ++i) inv[i] = -1;
    for (int m = kNs - 1; m >= 0; --m) {
        inv[kBins + m] = inv[lut[m]];
        inv[lut[m]] = (int16_t)m;
    }
}

uint64_t freq_key(double f) {
    uint64_t k;
    std::memcpy(&k, &f, sizeof k);
    return k;
}

// Index of the device table row for frequency f (uploaded on first use).
// Order in which the FP32 kernel's consumer threads take the 256 N-S beams:
// thread (TMEM lane ell, bin half hh) handles beam order[ell + 128 hh].  A warp
// gathers its 32 beams' bins from one shared-memory row with one 16-byte load
// per lane, eight consecutive lanes at a time; eight beams whose bins fall in
// distinct 16-byte bank groups (or that share a bin) load without a bank
// conflict, while the beams' natural order puts several bins of a group into
// one load.  Any order gives the same result.  Beams sharing a bin form units
// (at most eight beams); units are packed into the 32 groups of eight slots,
// largest first, by first fit and by best fit under a few orders of the units,
// and the packing with the fewest conflicts is kept (a conflict: one more
// distinct bin in a bank group of a slot group).
void gather_order(const int32_t* lut, int16_t* order) {
    constexpr int kOct = kNs / 8;
    struct Unit {
        int bin, group;
        std::vector<int> beams;
    };
    std::map<int, std::vector<int>> by_bin;
    for (int m = 0; m < kNs; ++m) by_bin[lut[m]].push_back(m);
    std::vector<Unit> units;
    for (auto& kv : by_bin) {
        const int L = kv.first, sw = L ^ ((L >> 3) & 1);     // the kernel's bin swizzle
        for (size_t i = 0; i < kv.second.size(); i += 8) {
            Unit u;
            u.bin = L;
            u.group = sw & 7;
            u.beams.assign(kv.second.begin() + i, kv.second.begin() + std::min(kv.second.size(), i + 8));
            units.push_back(std::move(u));
        }
    }
    auto conflicts = [&](const std::vector<std::vector<int>>& mem) {
        int extra = 0;
        for (const auto& o : mem) {
            std::map<int, std::set<int>> groups;
            for (int m : o) {
                const int L = lut[m];
                groups[(L ^ ((L >> 3) & 1)) & 7].insert(L);
            }
            int worst = 1;
            for (auto& g : groups) worst = std::max(worst, (int)g.second.size());
            extra += worst - 1;
        }
        return extra;
    };
    // one packing of the units in the given order; best = smallest room that fits
    auto pack = [&](const std::vector<int>& seq, bool best) {
        std::vector<std::vector<int>> mem(kOct);
        std::vector<std::map<int, int>> bin_of_group(kOct);     // group -> bin placed there
        for (int ui : seq) {
            const Unit& u = units[ui];
            const int n = (int)u.beams.size();
            auto fits = [&](int o, bool strict) {
                if ((int)mem[o].size() + n > 8) return false;
                if (!strict) return true;
                auto it = bin_of_group[o].find(u.group);
                return it == bin_of_group[o].end() || it->second == u.bin;
            };
            int pick = -1;
            for (int strict = 1; strict >= 0 && pick < 0; --strict)
                for (int o = 0; o < kOct; ++o)
                    if (fits(o, strict) && (pick < 0 || (best && mem[o].size() > mem[pick].size()))) {
                        pick = o;
                        if (!best) break;
                    }
            if (pick >= 0) {
                mem[pick].insert(mem[pick].end(), u.beams.begin(), u.beams.end());
                bin_of_group[pick].emplace(u.group, u.bin);
                continue;
            }
            for (int m : u.beams) {                        // split over whatever room is left
                int q = 0;
                while (mem[q].size() == 8) ++q;
                mem[q].push_back(m);
                bin_of_group[q].emplace(u.group, u.bin);
            }
        }
        return mem;
    };
    std::vector<int> seq(units.size());
    for (size_t i = 0; i < seq.size(); ++i) seq[i] = (int)i;
    auto by_size = [&](int a, int b) { return units[a].beams.size() > units[b].beams.size(); };
    std::vector<std::vector<int>> best_mem;
    int best_c = 1 << 30;
    uint32_t lcg = 12345u;
    for (int trial = 0; trial < 8 && best_c > 0; ++trial) {
        if (trial >= 2) {                                  // deterministic shuffles, then largest first
            for (size_t i = seq.size(); i > 1; --i) {
                lcg = lcg * 1664525u + 1013904223u;
                std::swap(seq[i - 1], seq[(lcg >> 8) % i]);
            }
        }
        std::stable_sort(seq.begin(), seq.end(), by_size);
        auto mem = pack(seq, (trial & 1) != 0);
        const int c = conflicts(mem);
        if (c < best_c) {
            best_c = c;
            best_mem = std::move(mem);
        }
    }
    int k = 0;
    for (const auto& o : best_mem)
        for (int m : o) order[k++] = (int16_t)m;
}

const unsigned char* tc_image(const bf_plan_s* p, int slot) {
    if (!p->terms) return nullptr;
    if (p->dft512) return p->d_a512;
    return p->atc_blocks[slot / kTcBlock] + (size_t)(slot % kTcBlock) * tc_a_bytes(p->terms);
}

// Slot holding the tables of frequency f, filled on first use (caller holds the lock).
// A new frequency takes a never-used slot while there is one, else the least
// recently used slot that no open stream and no unretired batch references.
int table_for(bf_plan_s* p, double f, int* idx) {
    const uint64_t key = freq_key(f);
    auto it = p->table_of_freq.find(key);
    if (it != p->table_of_freq.end()) {
        *idx = it->second;
        p->slot_used[*idx] = ++p->lru_clock;
        return BF_OK;
    }
    int n = -1;
    if (p->n_slots < p->table_cap) {
        n = p->n_slots;
    } else {
        for (int i = 0; i < p->table_cap; ++i)
            if (p->slot_refs[i] == 0 && (n < 0 || p->slot_used[i] < p->slot_used[n])) n = i;
        if (n < 0)
            return fail(BF_ENOMEM, "every per-frequency table slot is held by an open stream or a running batch "
                                   "(raise bf_config.max_tables)");
    }
    int32_t lut[kNs];
    int16_t lut16[kNs];
    float ew[2 * kEw * kCyl];
    clamp_table(p, f, lut);
    for (int m = 0; m < kNs; ++m) lut16[m] = (int16_t)lut[m];
    ew_table(p, f, ew);
    int16_t order[kNs];
    gather_order(lut, order);
    if (p->terms && !p->dft512) {
        const int blk = n / kTcBlock;
        if (!p->atc_blocks[blk]) CK(cudaMalloc(&p->atc_blocks[blk], (size_t)kTcBlock * tc_a_bytes(p->terms)));
    }
    // the slot is unreferenced: no launched kernel reads it, so plain copies can refill it
    if (n < p->n_slots) p->table_of_freq.erase(p->slot_key[n]);
    CK(cudaMemcpy(p->d_lut + (size_t)n * kNs, lut16, sizeof lut16, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->d_order + (size_t)n * kNs, order, sizeof order, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->d_ew + (size_t)n * kEw * kCyl, ew, sizeof ew, cudaMemcpyHostToDevice));
    if (p->dft512) {
        int16_t inv[kInvLen];
        inverse_clamp(lut, inv);
        CK(cudaMemcpy(p->d_inv + (size_t)n * kInvLen, inv, sizeof inv, cudaMemcpyHostToDevice));
    } else if (p->terms) {
        std::vector<__half> img;
        tc_image(p->terms, lut, kNs, img);
        CK(cudaMemcpy(const_cast<unsigned char*>(tc_image(p, n)), img.data(), img.size() * sizeof(__half),
                      cudaMemcpyHostToDevice));
    }
    if (n == p->n_slots) ++p->n_slots;
    p->slot_key[n] = key;
    p->slot_used[n] = ++p->lru_clock;
    p->table_of_freq[key] = n;
    *idx = n;
    return BF_OK;
}

// table_for plus one reference, for work that reads the slot outside the lock.
int hold_table(bf_plan_s* p, double f, int* idx) {
    int rc = table_for(p, f, idx);
    if (rc == BF_OK) ++p->slot_refs[*idx];
    return rc;
}

void release_table(bf_plan_s* p, int idx) {
    if (idx >= 0 && idx < (int)p->slot_refs.size() && p->slot_refs[idx] > 0) --p->slot_refs[idx];
}

// One reference on a table slot for the length of a synchronous inspection call.
struct TableHold {
    bf_plan_s* p;
    int idx = -1;
    explicit TableHold(bf_plan_s* plan) : p(plan) {}
    int take(double f) {
        std::lock_guard<std::mutex> lk(p->mu);
        return hold_table(p, f, &idx);
    }
    ~TableHold() {
        if (idx < 0) return;
        std::lock_guard<std::mutex> lk(p->mu);
        release_table(p, idx);
    }
};

Batch make_batch(const bf_plan_s* p) {
    Batch b;
    std::memset(&b, 0, sizeof b);
    b.lut = p->d_lut;
    b.inv = p->d_inv;
    b.order = p->d_order;
    b.ew = p->d_ew;
    b.tw512 = p->d_tw512;
    b.tw128 = p->d_tw128;
    b.status = p->d_status;
    b.part = p->d_part;
    b.part_tok = p->d_part_tok;
    b.park = p->d_park;
    return b;
}

int validate_request(const bf_request* r) {
    if (!r) return fail(BF_EINVAL, "null request");
    if (r->n_chan <= 0 || r->n_chan > 4096) return fail(BF_EINVAL, "n_chan out of range");
    if (r->n_samples < 0) return fail(BF_EINVAL, "negative n_samples");
    if (!r->chan_freq_hz) return fail(BF_EINVAL, "null chan_freq_hz");
    for (int c = 0; c < r->n_chan; ++c)
        if (!(r->chan_freq_hz[c] > 0.0) || !std::isfinite(r->chan_freq_hz[c]))
            return fail(BF_EINVAL, "channel frequency must be positive and finite");
    if (r->n_samples > 0 && !r->vin) return fail(BF_EINVAL, "null vin");
    if (((uintptr_t)r->vin & 15) != 0) return fail(BF_EINVAL, "vin must be 16-byte aligned");
    if (r->flags & ~BF_END_OF_STREAM) return fail(BF_EINVAL, "unknown flags");
    return BF_OK;
}

int64_t frames_for(const bf_plan_s* p, const bf_request* r, int carry_rows) {
    (void)p;
    return (carry_rows + r->n_samples) / kFrame;
}

size_t request_bytes(const bf_request* r, int64_t nf, bool new_stream) {
    size_t b = (size_t)r->n_chan * (size_t)r->n_samples * kInput;
    b += (size_t)kBeams * kSub * r->n_chan * (size_t)nf * sizeof(float);
    if (new_stream) b += (size_t)r->n_chan * (kFrame - 1) * kInput;
    return b;
}

// Carry buffer of `bytes` from the plan's pool (or a new allocation).  Buffers
// go back to the pool only after the batch that last used them has finished.
int carry_alloc(bf_plan_s* p, size_t bytes, uint8_t** out) {
    auto it = p->carry_pool.lower_bound(bytes);
    if (it != p->carry_pool.end() && it->first == bytes) {
        *out = it->second;
        p->carry_pool.erase(it);
        return BF_OK;
    }
    CK(cudaMalloc(out, bytes));
    return BF_OK;
}

// Stream state for a request (created on first use).  Caller holds the lock.
int stream_for(bf_plan_s* p, const bf_request* r, StreamState** out) {
    auto it = p->streams.find(r->stream_id);
    if (it != p->streams.end()) {
        if (it->second.n_chan != r->n_chan) return fail(BF_EINVAL, "stream changed its channel count");
        *out = &it->second;
        return BF_OK;
    }
    const int cap = p->cfg.max_streams > 0 ? p->cfg.max_streams : 1024;
    if ((int)p->streams.size() >= cap) return fail(BF_ENOMEM, "too many open streams");
    StreamState s;
    s.n_chan = r->n_chan;
    s.tables.resize(r->n_chan);
    for (int c = 0; c < r->n_chan; ++c) {
        // each channel's slot is referenced at once, so a later channel cannot evict it
        int rc = hold_table(p, r->chan_freq_hz[c], &s.tables[c]);
        if (rc) {
            for (int k = 0; k < c; ++k) release_table(p, s.tables[k]);
            return rc;
        }
    }
    s.carry_bytes = (size_t)r->n_chan * (kFrame - 1) * kInput;   // allocated when first needed
    auto res = p->streams.emplace(r->stream_id, std::move(s));
    *out = &res.first->second;
    return BF_OK;
}

// Enqueue one batch of jobs (one job per stream at most) on the plan stream:
// the fused kernel over all their frames, then the carry updates, then an
// event.  Caller holds the lock.  Returns BF_OK or an error.
int launch_jobs(bf_plan_s* p, std::vector<Job>& jobs, size_t bytes) {
    struct Carry {
        StreamState* st;
        const uint8_t* vin;
        int64_t n;
        int64_t nf;
        int old_rows;
        int new_rows;
        int n_chan;
        bool drop;
        uint64_t sid;
    };
    std::vector<Carry> carries;
    std::vector<Batch> batches;
    Batch b = make_batch(p);
    // tracking tables of this launch: one pinned staging buffer, one copy
    size_t track_elems = 0;
    for (auto& jb : jobs) track_elems += jb.track.size();
    TrackBuf tb;
    if (track_elems) {
        int rc = track_alloc(p, track_elems * sizeof(float2), &tb);
        if (rc) return rc;
    }
    size_t track_off = 0;
    // table slots the launches read, one reference each; an error before the first launch
    // drops them again (after it, a launched kernel may read them, so they stay held)
    std::vector<int> held;
    auto unhold = [&](int rc) {
        for (int t : held) release_table(p, t);
        if (tb.host) p->track_pool.emplace(tb.bytes, tb);
        return rc;
    };
    for (auto& jb : jobs) {
        StreamState* st = nullptr;
        int rc = stream_for(p, &jb.req, &st);
        if (rc) return unhold(rc);
        const int64_t nf = frames_for(p, &jb.req, st->carry_rows);
        const int new_rows = (int)((st->carry_rows + jb.req.n_samples) % kFrame);
        if (jb.track_frames >= 0 && jb.track_frames != nf)
            return unhold(fail(BF_EINVAL, "tracking table rows differ from the frames the request produces"));
        const float2* track_dev = nullptr;
        if (!jb.track.empty()) {
            std::memcpy(tb.host + track_off, jb.track.data(), jb.track.size() * sizeof(float2));
            track_dev = tb.dev + track_off;
            track_off += jb.track.size();
        }
        p->tickets[jb.ticket].n_frames = nf;
        for (int c = 0; c < jb.req.n_chan && nf > 0; ++c) {
            if (b.n_segs == kMaxSegs) {
                batches.push_back(b);
                b = make_batch(p);
            }
            Seg& s = b.segs[b.n_segs++];
            s.vin = jb.req.vin + (size_t)c * jb.req.n_samples * kInput;
            s.carry = st->carry ? st->carry + (size_t)c * (kFrame - 1) * kInput : nullptr;
            s.out = jb.req.out + (size_t)kSub * c * nf;
            s.beam_stride = (long long)kSub * jb.req.n_chan * nf;
            s.sub_stride = (int)nf;
            s.carry_rows = st->carry_rows;
            s.n_frames = (int)nf;
            s.table = st->tables[c];
            s.a_img = tc_image(p, s.table);
            held.push_back(s.table);
            ++p->slot_refs[s.table];
            s.ew_frames = track_dev ? track_dev + (size_t)c * nf * kEw * kCyl : nullptr;
            s.item_begin = b.n_items;
            b.n_items += (int)nf * kEw;
        }
        carries.push_back({st, jb.req.vin, jb.req.n_samples, nf, st->carry_rows, new_rows, jb.req.n_chan,
                           (jb.req.flags & BF_END_OF_STREAM) != 0, jb.req.stream_id});
        st->carry_rows = new_rows;      // host view advances at launch time
    }
    if (b.n_segs) batches.push_back(b);
    if (track_elems) {
        cudaError_t e = cudaMemcpyAsync(tb.dev, tb.host, track_elems * sizeof(float2), cudaMemcpyHostToDevice,
                                        p->stream);
        if (e != cudaSuccess) return unhold(cuda_fail(e, "tracking table upload"));
    }
    // timing events around the batch's device work, from the plan's pool (back to it on failure)
    struct PooledEvent {
        bf_plan_s* p;
        cudaEvent_t ev = nullptr;
        bool kept = false;
        ~PooledEvent() {
            if (ev && !kept) p->event_pool.push_back(ev);
        }
    } ev_start{p}, ev_end{p};
    for (PooledEvent* pe : {&ev_start, &ev_end}) {
        if (!p->event_pool.empty()) {
            pe->ev = p->event_pool.back();
            p->event_pool.pop_back();
        } else {
            CK(cudaEventCreate(&pe->ev));
        }
    }
    CK(cudaEventRecord(ev_start.ev, p->stream));
    for (auto& bb : batches) {
        bb.epoch = ++p->launches;
        // a launch of at most half a grid of items runs every item as two halves on two CTAs
        // (the 2-term tensor-core form never splits)
        cudaError_t e;
        if (p->dft512) {
            e = fused_tc_dft512_launch(bb, p->stream);
        } else if (p->terms == 1) {
            // the 1-term form runs on CTA pairs, one item per pair at a time
            e = fused_tc_pair_launch(bb, 2 * std::min(p->grid / 2, bb.n_items), p->stream);
        } else {
            int grid = std::min(p->grid, bb.n_items);
            if (p->terms != 2 && 2 * bb.n_items <= p->grid) grid = 2 * bb.n_items;
            e = p->terms ? fused_tc_launch(bb, p->terms, 0, grid, p->stream) : fused_fp32_launch(bb, grid, p->stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "fused kernel launch");
    }
    for (auto& c : carries) {
        if (c.drop) continue;
        int64_t src_row, dst_row, rows;
        if (c.nf > 0) {
            src_row = c.n - c.new_rows;
            dst_row = 0;
            rows = c.new_rows;
        } else {
            src_row = 0;
            dst_row = c.old_rows;
            rows = c.n;
        }
        if (rows > 0) {
            if (!c.st->carry) {
                int rc = carry_alloc(p, c.st->carry_bytes, &c.st->carry);
                if (rc) return rc;
            }
            CK(cudaMemcpy2DAsync(c.st->carry + dst_row * kInput, (size_t)(kFrame - 1) * kInput,
                                 c.vin + src_row * kInput, (size_t)c.n * kInput, (size_t)rows * kInput,
                                 c.n_chan, cudaMemcpyDeviceToDevice, p->stream));
        }
    }
    CK(cudaEventRecord(ev_end.ev, p->stream));
    ev_start.kept = ev_end.kept = true;
    InflightBatch ib{p->next_batch++, ev_end.ev, ev_start.ev, {}, bytes, {}, tb, std::move(held)};
    const double t_launch = now_s();
    for (auto& jb : jobs) {
        ib.tickets.push_back(jb.ticket);
        Ticket& t = p->tickets[jb.ticket];
        t.state = T_INFLIGHT;
        t.batch = ib.id;
        t.t_launch = t_launch;
    }
    for (auto& c : carries) {
        if (c.drop) {
            if (c.st->carry) ib.release.emplace_back(c.st->carry_bytes, c.st->carry);
            for (int t : c.st->tables) release_table(p, t);
            p->streams.erase(c.sid);
        }
    }
    p->inflight.push_back(std::move(ib));
    return BF_OK;
}

// Retire finished batches (caller holds the lock).  Returns true if any.
bool retire(bf_plan_s* p) {
    bool any = false;
    while (!p->inflight.empty()) {
        InflightBatch& ib = p->inflight.front();
        cudaError_t e = cudaEventQuery(ib.ev);
        if (e == cudaErrorNotReady) break;
        const bool expired = p->h_status && *(volatile int*)p->h_status != 0;
        if (expired) *(volatile int*)p->h_status = 0;
        const double t_done = now_s();
        float exec_ms = 0.f;
        if (e == cudaSuccess && cudaEventElapsedTime(&exec_ms, ib.ev_start, ib.ev) != cudaSuccess) exec_ms = 0.f;
        for (uint64_t t : ib.tickets) {
            auto it = p->tickets.find(t);
            if (it == p->tickets.end()) continue;
            it->second.t_done = t_done;
            it->second.t_exec = 1e-3 * exec_ms;
            if (e == cudaSuccess && expired) {
                it->second.state = T_ERROR;
                it->second.err = BF_ETIMEDOUT;
                it->second.msg = "a bounded device-side wait expired; the batch's output is incomplete";
            } else if (e == cudaSuccess) {
                it->second.state = T_DONE;
            } else {
                it->second.state = T_ERROR;
                it->second.err = BF_ECUDA;
                it->second.msg = std::string("batch failed: ") + cudaGetErrorString(e);
            }
        }
        p->mem_in_use -= std::min(p->mem_in_use, ib.bytes);
        for (auto& r : ib.release) p->carry_pool.emplace(r.first, r.second);
        if (ib.track.host) p->track_pool.emplace(ib.track.bytes, ib.track);
        for (int t : ib.slots) release_table(p, t);
        p->event_pool.push_back(ib.ev);
        p->event_pool.push_back(ib.ev_start);
        p->inflight.pop_front();
        any = true;
    }
    if (any) p->cv.notify_all();
    return any;
}

void worker_main(bf_plan_s* p) {
    cudaSetDevice(p->device);
    std::unique_lock<std::mutex> lk(p->mu);
    for (;;) {
        retire(p);
        // form the next batch: FIFO, one request per stream, within the budget
        std::vector<Job> jobs;
        size_t bytes = 0;
        int segs = 0;
        if ((int)p->inflight.size() < kMaxInflight) {
            std::vector<uint64_t> taken_streams;
            for (auto it = p->queue.begin(); it != p->queue.end();) {
                const uint64_t sid = it->req.stream_id;
                bool stream_seen = std::find(taken_streams.begin(), taken_streams.end(), sid) != taken_streams.end();
                // keep per-stream order: a stream blocked here blocks its later requests
                taken_streams.push_back(sid);
                if (stream_seen) {
                    ++it;
                    continue;
                }
                Ticket& t = p->tickets[it->ticket];
                const size_t budget = p->cfg.mem_budget;
                if ((budget && p->mem_in_use + bytes + t.bytes > budget) || segs + it->req.n_chan > 8 * kMaxSegs) {
                    ++it;
                    continue;
                }
                bytes += t.bytes;
                segs += it->req.n_chan;
                p->queued_bytes -= std::min(p->queued_bytes, t.bytes);
                jobs.push_back(std::move(*it));
                it = p->queue.erase(it);
            }
        }
        if (!jobs.empty()) {
            p->mem_in_use += bytes;
            int rc = launch_jobs(p, jobs, bytes);
            if (rc) {
                for (auto& jb : jobs) {
                    Ticket& t = p->tickets[jb.ticket];
                    t.state = T_ERROR;
                    t.err = rc;
                    t.msg = g_err;
                }
                p->mem_in_use -= std::min(p->mem_in_use, bytes);
                p->cv.notify_all();
            }
            continue;
        }
        if (p->stop && p->queue.empty() && p->inflight.empty()) break;
        if (p->inflight.empty())
            p->cv.wait(lk);
        else
            p->cv.wait_for(lk, std::chrono::microseconds(20));
    }
}

}  // namespace

extern "C" {

const char* bf_last_error(void) { return g_err.c_str(); }

int bf_config_default(bf_config* cfg) {
    if (!cfg) return fail(BF_EINVAL, "null config");
    std::memset(cfg, 0, sizeof *cfg);
    cfg->n_cyl = kCyl;
    cfg->n_feed = kFeed;
    cfg->n_pol = kPol;
    cfg->pad = kBins / kFeed;
    cfg->n_ew = kEw;
    cfg->upchan = kUp;
    cfg->f_ds = kFds;
    cfg->t_ds = kTds;
    cfg->feed_spacing_m = 0.3048;
    cfg->cyl_spacing_m = 20.0;
    cfg->dt_s = 2.56e-6;
    cfg->form = BF_FP32_FFT;
    cfg->mode = BF_MODE_DIRECT;
    cfg->device = -1;
    return BF_OK;
}

int bf_plan(const bf_config* cfg, bf_plan_t* out) {
    if (!cfg || !out) return fail(BF_EINVAL, "null argument");
    *out = nullptr;
    if (cfg->n_cyl != kCyl || cfg->n_feed != kFeed || cfg->n_pol != kPol || cfg->pad * kFeed != kBins ||
        cfg->n_ew != kEw || cfg->upchan != kUp || cfg->f_ds != kFds || cfg->t_ds != kTds)
        return fail(BF_EINVAL, "geometry differs from the one the kernels are built for (4x256x2, P=2, 4 E-W, 128/8/3)");
    if (!(cfg->feed_spacing_m > 0) || !(cfg->cyl_spacing_m >= 0) || !std::isfinite(cfg->feed_spacing_m) ||
        !std::isfinite(cfg->cyl_spacing_m))
        return fail(BF_EINVAL, "bad spacings");
    if (cfg->form != BF_FP32_FFT && cfg->form != BF_TC_DFT256 && cfg->form != BF_TC_DFT256_X2 &&
        cfg->form != BF_TC_DFT256_X1 && cfg->form != BF_TC_DFT512)
        return fail(BF_EINVAL, "unknown form");
    if (cfg->mode != BF_MODE_DIRECT && cfg->mode != BF_MODE_SERVING) return fail(BF_EINVAL, "bad mode");
    if (cfg->max_streams < 0) return fail(BF_EINVAL, "negative max_streams");
    if (cfg->max_tables < 0 || cfg->max_tables > kTableCap)
        return fail(BF_EINVAL, "max_tables must be 0 (default 4096) or 1 .. 4096");

    std::unique_ptr<bf_plan_s> p(new bf_plan_s);
    p->cfg = *cfg;
    p->terms = cfg->form == BF_TC_DFT256 ? 3 : cfg->form == BF_TC_DFT256_X2 ? 2 : cfg->form == BF_TC_DFT256_X1 ? 1 : 0;
    if (cfg->form == BF_TC_DFT512) {
        p->terms = 1;
        p->dft512 = true;
    }
    p->ns_sin.resize(kNs);
    p->ew_sin.resize(kEw);
    int prc = fill_pointings(p.get(), cfg);
    if (prc) return prc;
    p->cfg.ns_sin = nullptr;
    p->cfg.ew_sin = nullptr;

    if (cfg->device >= 0) {
        CK(cudaSetDevice(cfg->device));
        p->device = cfg->device;
    } else {
        CK(cudaGetDevice(&p->device));
    }
    int major = 0, minor = 0;
    CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, p->device));
    CK(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, p->device));
    if (major != 10 || minor != 3)
        return fail(BF_EINVAL, "this library is built for sm_103a (GB300) only; device is sm_" +
                                   std::to_string(major) + std::to_string(minor));
    p->grid = fused_fp32_max_grid(p->device);
    if (p->grid <= 0) return fail(BF_ECUDA, "cannot query SM count");

    if (cfg->cuda_stream) {
        p->stream = (cudaStream_t)cfg->cuda_stream;
    } else {
        CK(cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking));
        p->own_stream = true;
    }
    p->table_cap = cfg->max_tables > 0 ? cfg->max_tables : kTableCap;
    p->slot_key.assign(p->table_cap, 0);
    p->slot_refs.assign(p->table_cap, 0);
    p->slot_used.assign(p->table_cap, 0);
    p->atc_blocks.assign((p->table_cap + kTcBlock - 1) / kTcBlock, nullptr);
    CK(cudaMalloc(&p->d_lut, (size_t)p->table_cap * kNs * sizeof(int16_t)));
    CK(cudaMalloc(&p->d_order, (size_t)p->table_cap * kNs * sizeof(int16_t)));
    CK(cudaMalloc(&p->d_ew, (size_t)p->table_cap * kEw * kCyl * sizeof(float2)));
    CK(cudaMalloc(&p->d_tw512, kBins * sizeof(float2)));
    CK(cudaMalloc(&p->d_tw128, kUp * sizeof(float2)));
    if (p->dft512) {
        CK(cudaMalloc(&p->d_inv, (size_t)p->table_cap * kInvLen * sizeof(int16_t)));
        int32_t all[kBins];
        for (int k = 0; k < kBins; ++k) all[k] = k;
        std::vector<__half> img;
        tc_image(1, all, kBins, img);
        CK(cudaMalloc(&p->d_a512, img.size() * sizeof(__half)));
        CK(cudaMemcpy(p->d_a512, img.data(), img.size() * sizeof(__half), cudaMemcpyHostToDevice));
    }
    std::vector<float2> tw(kBins);
    for (int e = 0; e < kBins; ++e)
        tw[e] = make_float2((float)std::cos(-2.0 * kPi * e / kBins), (float)std::sin(-2.0 * kPi * e / kBins));
    CK(cudaMemcpy(p->d_tw512, tw.data(), kBins * sizeof(float2), cudaMemcpyHostToDevice));
    for (int e = 0; e < kUp; ++e)
        tw[e] = make_float2((float)std::cos(-2.0 * kPi * e / kUp), (float)std::sin(-2.0 * kPi * e / kUp));
    CK(cudaMemcpy(p->d_tw128, tw.data(), kUp * sizeof(float2), cudaMemcpyHostToDevice));
    CK(cudaHostAlloc(&p->h_status, sizeof(int), cudaHostAllocMapped));
    *p->h_status = 0;
    CK(cudaHostGetDevicePointer(&p->d_status, p->h_status, 0));
    if (p->grid <= 2 * kMaxSplit) {
        // a launch splits at most grid / 2 items: two halves of 16 x 256 floats each, and
        // one token per bin; the tensor-core form also parks each CTA's first half
        const size_t slots = (size_t)p->grid / 2 + 1;
        CK(cudaMalloc(&p->d_part, slots * 2 * kSub * kNs * sizeof(float)));
        CK(cudaMalloc(&p->d_part_tok, slots * kNs * sizeof(unsigned long long)));
        CK(cudaMemset(p->d_part_tok, 0, slots * kNs * sizeof(unsigned long long)));
        if (p->terms) CK(cudaMalloc(&p->d_park, (size_t)p->grid * kSub * kNs * sizeof(float)));
    }

    if (p->cfg.mode == BF_MODE_SERVING) {
        bf_plan_s* raw = p.get();
        raw->worker = std::thread(worker_main, raw);
    }
    *out = p.release();
    return BF_OK;
}

int bf_frames_out(bf_plan_t p, uint64_t stream_id, int64_t n_samples, int64_t* n_frames_out) {
    if (!p || !n_frames_out || n_samples < 0) return fail(BF_EINVAL, "bad argument");
    std::lock_guard<std::mutex> lk(p->mu);
    int carry = 0;
    auto it = p->streams.find(stream_id);
    if (it != p->streams.end()) carry = it->second.carry_rows;
    // queued requests of this stream advance the carry too
    for (auto& jb : p->queue)
        if (jb.req.stream_id == stream_id) carry = (int)((carry + jb.req.n_samples) % kFrame);
    *n_frames_out = (carry + n_samples) / kFrame;
    return BF_OK;
}

int bf_submit(bf_plan_t p, const bf_request* r, uint64_t* ticket) {
    if (!p || !ticket) return fail(BF_EINVAL, "null argument");
    int rc = validate_request(r);
    if (rc) return rc;
    CK(cudaSetDevice(p->device));
    std::unique_lock<std::mutex> lk(p->mu);
    if (p->stop) return fail(BF_ESHUTDOWN, "plan is shutting down");
    auto sit = p->streams.find(r->stream_id);
    if (sit != p->streams.end() && sit->second.n_chan != r->n_chan)
        return fail(BF_EINVAL, "stream changed its channel count");
    if (r->n_samples > 0 && !r->out) {
        int carry = sit != p->streams.end() ? sit->second.carry_rows : 0;
        for (auto& jb : p->queue)
            if (jb.req.stream_id == r->stream_id) carry = (int)((carry + jb.req.n_samples) % kFrame);
        if ((carry + r->n_samples) / kFrame > 0) return fail(BF_EINVAL, "null out with frames to write");
    }
    Job jb;
    if (r->ew_sin_frames) {
        // frames this request produces: the stream's carry advanced by its queued requests
        int carry = sit != p->streams.end() ? sit->second.carry_rows : 0;
        for (auto& q : p->queue)
            if (q.req.stream_id == r->stream_id) carry = (int)((carry + q.req.n_samples) % kFrame);
        const int64_t nf = (carry + r->n_samples) / kFrame;
        for (int64_t i = 0; i < nf * kEw; ++i)
            if (!std::isfinite(r->ew_sin_frames[i]) || std::fabs(r->ew_sin_frames[i]) > 1.0)
                return fail(BF_EINVAL, "tracking E-W sines must be finite and within [-1, 1]");
        jb.track_frames = nf;
        jb.track.resize((size_t)r->n_chan * nf * kEw * kCyl);
        for (int c = 0; c < r->n_chan; ++c)
            for (int64_t F = 0; F < nf; ++F)
                ew_phases(p, r->chan_freq_hz[c], r->ew_sin_frames + F * kEw,
                          reinterpret_cast<float*>(jb.track.data() + ((size_t)c * nf + F) * kEw * kCyl));
    }
    jb.ticket = p->next_ticket++;
    jb.req = *r;
    jb.req.ew_sin_frames = nullptr;
    jb.freqs.assign(r->chan_freq_hz, r->chan_freq_hz + r->n_chan);
    jb.req.chan_freq_hz = jb.freqs.data();
    Ticket t;
    t.t_submit = now_s();
    t.bytes = request_bytes(r, (int64_t)(r->n_samples / kFrame) + 1, sit == p->streams.end());
    if (p->cfg.mem_budget && t.bytes > p->cfg.mem_budget)
        return fail(BF_ENOMEM, "request larger than the plan's memory budget");
    p->tickets[jb.ticket] = t;
    *ticket = jb.ticket;

    if (p->cfg.mode == BF_MODE_DIRECT) {
        std::vector<Job> jobs;
        jobs.push_back(std::move(jb));
        rc = launch_jobs(p, jobs, 0);
        if (rc) {
            p->tickets.erase(*ticket);
            return rc;
        }
        return BF_OK;
    }
    // admitted at once only if it fits beside everything launched or queued before it
    const bool fits = !p->cfg.mem_budget || p->mem_in_use + p->queued_bytes + t.bytes <= p->cfg.mem_budget;
    p->queued_bytes += t.bytes;
    p->queue.push_back(std::move(jb));
    p->cv.notify_all();
    return fits ? BF_OK : BF_EQUEUED;
}

static int poll_ticket(bf_plan_t p, uint64_t ticket, int64_t timeout_us, int64_t* n_frames_out, double* times) {
    if (!p) return fail(BF_EINVAL, "null plan");
    const auto t0 = std::chrono::steady_clock::now();
    std::unique_lock<std::mutex> lk(p->mu);
    for (;;) {
        auto it = p->tickets.find(ticket);
        if (it == p->tickets.end()) return fail(BF_ENOTICKET, "unknown ticket");
        if (it->second.state == T_INFLIGHT) retire(p);
        it = p->tickets.find(ticket);
        if ((it->second.state == T_DONE || it->second.state == T_ERROR) && times) {
            times[0] = it->second.t_submit;
            times[1] = it->second.t_launch;
            times[2] = it->second.t_done;
            times[3] = now_s();
            times[4] = it->second.t_exec;
        }
        if (it->second.state == T_DONE) {
            if (n_frames_out) *n_frames_out = it->second.n_frames;
            p->tickets.erase(it);
            return BF_OK;
        }
        if (it->second.state == T_ERROR) {
            int err = it->second.err;
            g_err = it->second.msg;
            p->tickets.erase(it);
            return err;
        }
        const auto el = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
        if (timeout_us >= 0 && el >= timeout_us) return BF_PENDING;
        // inflight: poll the event; queued: wait for the worker
        p->cv.wait_for(lk, std::chrono::microseconds(it->second.state == T_INFLIGHT ? 10 : 200));
    }
}

int bf_poll(bf_plan_t p, uint64_t ticket, int64_t timeout_us, int64_t* n_frames_out) {
    return poll_ticket(p, ticket, timeout_us, n_frames_out, nullptr);
}

int bf_poll_timed(bf_plan_t p, uint64_t ticket, int64_t timeout_us, int64_t* n_frames_out, double* times) {
    if (!times) return fail(BF_EINVAL, "null times");
    return poll_ticket(p, ticket, timeout_us, n_frames_out, times);
}

int bf_destroy(bf_plan_t p) {
    if (!p) return fail(BF_EINVAL, "null plan");
    cudaSetDevice(p->device);
    {
        std::lock_guard<std::mutex> lk(p->mu);
        p->stop = true;
        p->cv.notify_all();
    }
    if (p->worker.joinable()) p->worker.join();
    int rc = BF_OK;
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
    {
        std::lock_guard<std::mutex> lk(p->mu);
        retire(p);
        for (auto& kv : p->streams)
            if (kv.second.carry) cudaFree(kv.second.carry);
        for (auto& ib : p->inflight) {
            cudaEventDestroy(ib.ev);
            cudaEventDestroy(ib.ev_start);
            for (auto& r : ib.release) cudaFree(r.second);
            if (ib.track.host) p->track_pool.emplace(ib.track.bytes, ib.track);
        }
        for (auto& kv : p->carry_pool) cudaFree(kv.second);
        for (auto& kv : p->track_pool) {
            cudaFreeHost(kv.second.host);
            cudaFree(kv.second.dev);
        }
        for (auto ev : p->event_pool) cudaEventDestroy(ev);
    }
    cudaFree(p->d_lut);
    cudaFree(p->d_order);
    cudaFree(p->d_ew);
    cudaFree(p->d_tw512);
    cudaFree(p->d_tw128);
    cudaFree(p->d_part);
    cudaFree(p->d_part_tok);
    cudaFree(p->d_park);
    cudaFree(p->d_inv);
    cudaFree(p->d_a512);
    for (unsigned char* blk : p->atc_blocks)
        if (blk) cudaFree(blk);
    if (p->d_delays) cudaFree(p->d_delays);
    if (p->h_status) cudaFreeHost(p->h_status);
    if (p->own_stream) cudaStreamDestroy(p->stream);
    delete p;
    return rc;
}

// ---- products of the intensity output -------------------------------------------------------

int bf_skymap(bf_plan_t p, const float* d_out, int64_t n_sub, int64_t n_frames, float* d_map) {
    if (!p || n_sub < 0 || n_frames < 0 || !d_map || (n_sub * n_frames > 0 && !d_out))
        return fail(BF_EINVAL, "bad argument");
    CK(cudaSetDevice(p->device));
    CK(skymap_launch(d_out, kBeams, (long long)(n_sub * n_frames), d_map, p->stream));
    return BF_OK;
}

}  // extern "C"

namespace {

// Dedispersion delays in frames of every sub-channel (rule of bf_dedisperse);
// d must hold kSub * n_chan entries.  Returns BF_OK or BF_EINVAL.
int dedisperse_delays(int n_chan, const double* chan_freq_hz, double dm, int* d, int* dmax_out) {
    const int n_sub = kSub * n_chan;
    const double fine = 390625.0 / kUp;
    double fmax = 0.0;
    for (int c = 0; c < n_chan; ++c) {
        if (!(chan_freq_hz[c] > 0) || !std::isfinite(chan_freq_hz[c])) return fail(BF_EINVAL, "bad frequency");
        for (int s = 0; s < kSub; ++s)
            fmax = std::max(fmax, (chan_freq_hz[c] + (kFds * s + (kFds - 1) / 2.0 - kUp / 2) * fine) / 1e6);
    }
    int dmax = 0;
    for (int i = 0; i < n_sub; ++i) {
        const int c = i / kSub, s = i % kSub;
        const double f = (chan_freq_hz[c] + (kFds * s + (kFds - 1) / 2.0 - kUp / 2) * fine) / 1e6;
        const double x = ((4.148808e3 * dm) * (1.0 / (f * f) - 1.0 / (fmax * fmax))) / (kFrame * 2.56e-6);
        d[i] = (int)std::floor(x + 0.5);
        dmax = std::max(dmax, d[i]);
    }
    *dmax_out = dmax;
    return BF_OK;
}

}  // namespace

extern "C" {

int bf_dedisperse(bf_plan_t p, const float* d_out, int n_chan, const double* chan_freq_hz, int64_t n_frames,
                  double dm, float* d_series, int64_t* n_out) {
    if (!p || n_chan <= 0 || n_chan > 4096 || !chan_freq_hz || n_frames < 0 || !n_out || !(dm >= 0) ||
        !std::isfinite(dm))
        return fail(BF_EINVAL, "bad argument");
    const int n_sub = kSub * n_chan;
    std::vector<int> d(n_sub);
    int dmax = 0;
    int rc = dedisperse_delays(n_chan, chan_freq_hz, dm, d.data(), &dmax);
    if (rc) return rc;
    *n_out = std::max<int64_t>(0, n_frames - dmax);
    if (*n_out == 0) return BF_OK;
    if (!d_out || !d_series) return fail(BF_EINVAL, "null buffer");
    CK(cudaSetDevice(p->device));
    std::lock_guard<std::mutex> lk(p->mu);
    if (p->delays_cap < (size_t)n_sub) {
        if (p->d_delays) CK(cudaFree(p->d_delays));
        p->d_delays = nullptr;
        CK(cudaMalloc(&p->d_delays, (size_t)n_sub * sizeof(int)));
        p->delays_cap = n_sub;
    }
    // pageable source: the copy is staged before the call returns, in stream order
    CK(cudaMemcpyAsync(p->d_delays, d.data(), (size_t)n_sub * sizeof(int), cudaMemcpyHostToDevice, p->stream));
    CK(dedisperse_launch(d_out, p->d_delays, n_sub, (long long)n_frames, (long long)*n_out, d_series, p->stream));
    return BF_OK;
}

int bf_dedisperse_static(bf_plan_t p, const float* d_out, int n_chan, const double* chan_freq_hz,
                         int64_t n_frames, double dm, float* d_series, int64_t* n_out) {
    if (!p || n_chan <= 0 || !chan_freq_hz || n_frames < 0 || !n_out || !(dm >= 0) || !std::isfinite(dm))
        return fail(BF_EINVAL, "bad argument");
    if (n_chan > kDdStaticMaxSub / kSub)         // checked before any product, so no overflow
        return fail(BF_EINVAL, "more channels than the static delay table holds (4096 channels, 65536 sub-channels)");
    const int n_sub = kSub * n_chan;
    std::vector<int> d(n_sub);
    int dmax = 0;
    int rc = dedisperse_delays(n_chan, chan_freq_hz, dm, d.data(), &dmax);
    if (rc) return rc;
    *n_out = std::max<int64_t>(0, n_frames - dmax);
    if (*n_out == 0) return BF_OK;
    if (!d_out || !d_series) return fail(BF_EINVAL, "null buffer");
    CK(cudaSetDevice(p->device));
    int* table = nullptr;
    CK(dedisperse_static_table(p->device, &table));
    CK(cudaMemcpyAsync(table, d.data(), (size_t)n_sub * sizeof(int), cudaMemcpyHostToDevice, p->stream));
    CK(dedisperse_launch(d_out, table, n_sub, (long long)n_frames, (long long)*n_out, d_series, p->stream));
    return BF_OK;
}


int bf_rescale_u8(bf_plan_t p, const float* d_out, int64_t n_rows, int64_t n_frames, uint8_t* d_codes,
                  float* d_stats) {
    if (!p || n_rows < 0 || n_frames < 0 || (n_rows * n_frames > 0 && (!d_out || !d_codes)))
        return fail(BF_EINVAL, "bad argument");
    CK(cudaSetDevice(p->device));
    CK(rescale_u8_launch(d_out, (long long)n_rows, (long long)n_frames, d_codes, d_stats, p->stream));
    return BF_OK;
}

// ---- inspection entry points ------------------------------------------------------------

int bf_debug_tables(const bf_config* cfg, double freq_hz, int32_t* lut_out, float* ew_out) {
    if (!cfg || !(freq_hz > 0) || !std::isfinite(freq_hz)) return fail(BF_EINVAL, "bad argument");
    bf_plan_s tmp;
    tmp.cfg = *cfg;
    tmp.ns_sin.resize(kNs);
    tmp.ew_sin.resize(kEw);
    int rc = fill_pointings(&tmp, cfg);
    if (rc) return rc;
    if (lut_out) clamp_table(&tmp, freq_hz, lut_out);
    if (ew_out) ew_table(&tmp, freq_hz, ew_out);
    return BF_OK;
}

int bf_debug_gather_order(const bf_config* cfg, double freq_hz, int16_t* order_out) {
    if (!cfg || !order_out || !(freq_hz > 0) || !std::isfinite(freq_hz)) return fail(BF_EINVAL, "bad argument");
    bf_plan_s tmp;
    tmp.cfg = *cfg;
    tmp.ns_sin.resize(kNs);
    tmp.ew_sin.resize(kEw);
    int rc = fill_pointings(&tmp, cfg);
    if (rc) return rc;
    int32_t lut[kNs];
    clamp_table(&tmp, freq_hz, lut);
    gather_order(lut, order_out);
    return BF_OK;
}

int bf_debug_unpack(bf_plan_t p, const uint8_t* d_in, float* d_out, int64_t n) {
    if (!p || n < 0 || (n > 0 && (!d_in || !d_out))) return fail(BF_EINVAL, "bad argument");
    CK(cudaSetDevice(p->device));
    CK(debug_unpack_launch(d_in, d_out, n, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    return BF_OK;
}

int bf_debug_beams(bf_plan_t p, double freq_hz, const uint8_t* d_vin, int64_t n_samples, float* d_out) {
    if (!p || n_samples < 0 || !(freq_hz > 0) || (n_samples > 0 && (!d_vin || !d_out)))
        return fail(BF_EINVAL, "bad argument");
    if (((uintptr_t)d_vin & 15) != 0) return fail(BF_EINVAL, "vin must be 16-byte aligned");
    CK(cudaSetDevice(p->device));
    TableHold hold(p);
    int rc = hold.take(freq_hz);
    if (rc) return rc;
    const int tab = hold.idx;
    CK(debug_beams_launch(d_vin, n_samples, p->d_lut + (size_t)tab * kNs, p->d_ew + (size_t)tab * kEw * kCyl,
                          p->d_tw512, reinterpret_cast<float2*>(d_out), p->stream));
    CK(cudaStreamSynchronize(p->stream));
    return BF_OK;
}

static int debug_fused(bf_plan_t p, double freq_hz, const uint8_t* d_vin, int64_t n_samples, float* d_out,
                       int mode) {
    if (!p || n_samples < 0 || n_samples % kFrame != 0 || !(freq_hz > 0) || (n_samples > 0 && (!d_vin || !d_out)))
        return fail(BF_EINVAL, "bad argument (n_samples must be a multiple of 384)");
    if (((uintptr_t)d_vin & 15) != 0) return fail(BF_EINVAL, "vin must be 16-byte aligned");
    if (mode == 2 && !p->terms) return fail(BF_EINVAL, "the GEMM dump needs a tensor-core form");
    if (p->dft512) return fail(BF_EINVAL, "stage dumps are not built for the 512-row form");
    CK(cudaSetDevice(p->device));
    Batch b = make_batch(p);
    TableHold hold(p);
    int rc = hold.take(freq_hz);
    if (rc) return rc;
    b.segs[0].table = hold.idx;
    b.segs[0].a_img = tc_image(p, hold.idx);
    const int nf = (int)(n_samples / kFrame);
    b.n_segs = 1;
    b.n_items = nf * kEw;
    b.segs[0].vin = d_vin;
    b.segs[0].n_frames = nf;
    b.dump = reinterpret_cast<float2*>(d_out);
    const int grid = std::min(p->grid, std::max(b.n_items, 1));
    if (p->terms) {
        CK(fused_tc_launch(b, p->terms, mode, grid, p->stream));
    } else {
        CK(fused_fp32_dump_launch(b, grid, p->stream));
    }
    CK(cudaStreamSynchronize(p->stream));
    if (p->h_status && *(volatile int*)p->h_status) {
        *(volatile int*)p->h_status = 0;
        return fail(BF_ETIMEDOUT, "a bounded device-side wait expired");
    }
    return BF_OK;
}

int bf_debug_upchan(bf_plan_t p, double freq_hz, const uint8_t* d_vin, int64_t n_samples, float* d_out) {
    return debug_fused(p, freq_hz, d_vin, n_samples, d_out, 1);
}

int bf_debug_gemm(bf_plan_t p, double freq_hz, const uint8_t* d_vin, int64_t n_samples, float* d_out) {
    return debug_fused(p, freq_hz, d_vin, n_samples, d_out, 2);
}

int bf_debug_stall(bf_plan_t p, const uint8_t* d_vin, int64_t wait_ns) {
    if (!p || !d_vin || wait_ns <= 0 || wait_ns > 2000000000LL) return fail(BF_EINVAL, "bad argument");
    if (((uintptr_t)d_vin & 15) != 0) return fail(BF_EINVAL, "vin must be 16-byte aligned");
    CK(cudaSetDevice(p->device));
    Batch b = make_batch(p);
    TableHold hold(p);
    int rc = hold.take(600e6);
    if (rc) return rc;
    b.segs[0].table = hold.idx;
    b.segs[0].a_img = tc_image(p, hold.idx);
    b.n_segs = 1;
    b.n_items = kEw;                       // one frame, four E-W beams
    b.segs[0].vin = d_vin;
    b.segs[0].n_frames = 1;
    b.wait_ns = (unsigned long long)wait_ns;
    if (p->dft512 || p->terms == 1) {
        // the form's own kernel: clusters of four (512 rows) or two (256 rows, 1 term)
        CK(fused_tc_pair_stall_launch(b, p->dft512 ? 4 : 2, p->stream));
    } else {
        CK(fused_tc_launch(b, 1, 3, std::min(p->grid, kEw), p->stream));
    }
    CK(cudaStreamSynchronize(p->stream));
    if (p->h_status && *(volatile int*)p->h_status) {
        *(volatile int*)p->h_status = 0;
        return fail(BF_ETIMEDOUT, "a bounded device-side wait expired (expected in the stall check)");
    }
    return BF_OK;
}

// ---- measurement aid ---------------------------------------------------------------------

int bf_fp32_fma_probe(void* cuda_stream, int paired, int64_t iters, float* d_sink, int64_t n_sink, double* flop_out) {
    if (iters <= 0 || !d_sink || n_sink < 256 || !flop_out) return fail(BF_EINVAL, "bad argument");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(fma_probe_launch(paired != 0, (long long)iters, d_sink, (long long)n_sink, sms, flop_out,
                        (cudaStream_t)cuda_stream));
    return BF_OK;
}

}  // extern "C"
