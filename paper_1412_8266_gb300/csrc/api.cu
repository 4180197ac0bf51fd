// C ABI entry points (srng.h): stream sets, jumps, generation, state I/O.
//
// Host side of the paper's initialisation layer (arXiv 1412.8266 Sec. 5.1):
// one call allocates the device state and places every stream before any
// user kernel runs; the device never sees host-only concepts.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "srng.h"

namespace srng_impl {

// ------------------------------------------------------------------ errors
namespace {
thread_local std::string t_last_error;
}

srng_status fail(srng_status st, const std::string &msg)
{
    t_last_error = msg;
    return st;
}

srng_status cuda_fail(cudaError_t e, const char *what)
{
    t_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? SRNG_ERR_OOM : SRNG_ERR_CUDA;
}

void clear_error() { t_last_error.clear(); }

// ------------------------------------------------------------------ devices
srng_status current_device(DeviceInfo *out)
{
    static std::mutex mu;
    static std::map<int, int> sm_counts;
    int dev = 0;
    SRNG_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    auto it = sm_counts.find(dev);
    if (it == sm_counts.end()) {
        int sms = 0;
        SRNG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        it = sm_counts.emplace(dev, sms).first;
    }
    out->device = dev;
    out->sm_count = it->second;
    return SRNG_OK;
}

// ------------------------------------------------------------------ tuning
namespace {
std::mutex g_tune_mu;
srng_tune g_tune[3][3];   // rows: MRG32k3a, counter-based (Philox, Threefry), TinyMT32
bool g_tune_set[3][3];

srng_tune builtin_tune(srng_gen gen, srng_out type)
{
    srng_tune t;
    memset(&t, 0, sizeof t);
    t.block_threads = 256;
    // counter-based generators: grids of 16 blocks per SM, more than fit at
    // once, handed out by the block scheduler as blocks finish (2^18 streams
    // x 4096 words 0.861 -> 0.840 ms, 2^30 words 0.673 -> 0.666 ms against 8)
    t.blocks_per_sm = tune_row(gen) == 1 ? 16 : 8;
    t.chunk = 0;  // chosen from the problem shape
    // the fused variates carry long single-precision sequences: one block pair
    // per lane keeps the registers (and the resident warps) of the uniforms;
    // doubles: two pairs (2^30 Philox doubles 1.20 ms, against 1.28 with four)
    t.unroll = type == SRNG_OUT_EXP_F32 || type == SRNG_OUT_NORMAL_F32 ? 1 : type == SRNG_OUT_F64 ? 2 : 4;
    // MRG32k3a whole-row items: doubles from each lane's registers with 32-byte
    // stores, three in eight through the FP64 multiply; 4-byte values through
    // the shared-memory row stage (the measured best of each at 2^18 x 4096),
    // or, for streams cut into a multiple of 32 chunks (radix-32 chunk starts),
    // from each lane's registers (0: decided by the call's shape; 64 x 2^16
    // uint32 11.3 us per call against 13.4 staged)
    t.vector_store = gen == SRNG_MRG32K3A ? (type == SRNG_OUT_F64 ? 4 : 0) : 1;
    // the FP64 direct rows run best with 6 or 7 resident blocks of 256 per SM
    // (2^18 x 4096: 1.75 ms, against 1.88 with the 8 its registers allow)
    t.resident = gen == SRNG_MRG32K3A && type == SRNG_OUT_F64 ? 6 : 0;
    t.lane_blocks = 64;
    return t;
}
}  // namespace

srng_tune effective_tune(srng_gen gen, srng_out type, const srng_tune *user)
{
    gen = (srng_gen)kernel_gen(gen);
    srng_tune t = builtin_tune(gen, type);
    const int row = tune_row(gen);
    const int col = type == SRNG_OUT_F64 ? SRNG_OUT_F64 : type == SRNG_OUT_U32 ? SRNG_OUT_U32 : SRNG_OUT_F32;
    {   // the fused variate outputs take the FP32 entries
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (g_tune_set[row][col]) {
            const srng_tune &d = g_tune[row][col];
            if (d.block_threads) t.block_threads = d.block_threads;
            if (d.blocks_per_sm) t.blocks_per_sm = d.blocks_per_sm;
            if (d.chunk) t.chunk = d.chunk;
            if (d.unroll) t.unroll = d.unroll;
            if (d.vector_store) t.vector_store = d.vector_store;
            if (d.lane_blocks) t.lane_blocks = d.lane_blocks;
            if (d.resident) t.resident = d.resident;
        }
    }
    if (user) {
        if (user->block_threads) t.block_threads = user->block_threads;
        if (user->blocks_per_sm) t.blocks_per_sm = user->blocks_per_sm;
        if (user->chunk) t.chunk = user->chunk;
        if (user->unroll) t.unroll = user->unroll;
        if (user->vector_store) t.vector_store = user->vector_store;
        if (user->lane_blocks) t.lane_blocks = user->lane_blocks;
        if (user->resident) t.resident = user->resident;
    }
    return t;
}

srng_status check_tune(const srng_tune *t)
{
    if (!t) return SRNG_OK;
    if (t->block_threads && (t->block_threads % 32 || t->block_threads > 256 || t->block_threads < 64))
        return fail(SRNG_ERR_ARG, "tune.block_threads must be a multiple of 32 in [64, 256]");
    if (t->blocks_per_sm > 64) return fail(SRNG_ERR_ARG, "tune.blocks_per_sm must be <= 64");
    if (t->chunk && t->chunk % 32) return fail(SRNG_ERR_ARG, "tune.chunk must be a multiple of 32");
    if (t->unroll && t->unroll != 1 && t->unroll != 2 && t->unroll != 4)
        return fail(SRNG_ERR_ARG, "tune.unroll must be 1, 2 or 4");
    if (t->vector_store > 4) return fail(SRNG_ERR_ARG, "tune.vector_store must be 0, 1, 2, 3 or 4");
    if (t->lane_blocks > 4096) return fail(SRNG_ERR_ARG, "tune.lane_blocks must be <= 4096");
    if (t->resident > 32) return fail(SRNG_ERR_ARG, "tune.resident must be <= 32");
    return SRNG_OK;
}

// --------------------------------------------------------- jump tables
namespace {
std::mutex g_tab_mu;
std::map<std::pair<int, uint64_t>, JumpTable> g_tabs;  // (shift, chunk) -> J_k = A^(chunk 2^(shift+k))

// J_k = (A^(base * 2^shift))^(2^k), k < 64.
const JumpTable &jump_table(int shift, uint64_t base)
{
    std::lock_guard<std::mutex> lk(g_tab_mu);
    auto key = std::make_pair(shift, base);
    auto it = g_tabs.find(key);
    if (it != g_tabs.end()) return it->second;
    JumpTable t;
    MatPair m = mat_pow_shifted(0, base, shift);
    for (int k = 0; k < 64; ++k) {
        memcpy(t.m[k], m.a, sizeof m.a);
        m = mat_mul(m, m);
    }
    return g_tabs.emplace(key, t).first->second;
}

std::map<uint64_t, RadixTable> g_radix;  // chunk -> A^(chunk l), A^(32 chunk g)

const RadixTable &radix_table(uint64_t chunk)
{
    std::lock_guard<std::mutex> lk(g_tab_mu);
    auto it = g_radix.find(chunk);
    if (it != g_radix.end()) return it->second;
    RadixTable r;
    const MatPair c = mat_pow_shifted(0, chunk, 0);
    MatPair m = mat_identity();
    for (int l = 0; l < 32; ++l) {
        memcpy(r.lane[l], m.a, sizeof m.a);
        m = mat_mul(m, c);
    }
    const MatPair w = m;  // A^(32 chunk)
    m = mat_identity();
    for (int g = 0; g < 32; ++g) {
        memcpy(r.warp[g], m.a, sizeof m.a);
        m = mat_mul(m, w);
    }
    return g_radix.emplace(chunk, r).first->second;
}

int bit_length(uint64_t x)
{
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

size_t out_size(srng_out t) { return t == SRNG_OUT_F64 ? 8 : 4; }

bool valid_gen(int g)
{
    return g == SRNG_MRG32K3A || g == SRNG_PHILOX4X32_10 || g == SRNG_PHILOX4X32_10_KEYED ||
           g == SRNG_THREEFRY4X32_20 || g == SRNG_TINYMT32 || g == SRNG_THREEFRY4X64_20;
}
bool valid_out(int t) { return t == SRNG_OUT_U32 || t == SRNG_OUT_F32 || t == SRNG_OUT_F64; }
// Output types of the bulk generation calls (the uniforms and the fused variates).
bool valid_gen_out(int t) { return valid_out(t) || t == SRNG_OUT_EXP_F32 || t == SRNG_OUT_NORMAL_F32; }

int spacing_shift(srng_spacing sp) { return sp == SRNG_SPACING_SUBSTREAM ? 76 : 127; }

}  // namespace

// Placement of streams [first, first + count) of an MRG32k3a set.
static srng_status place_streams(srng_set *s, uint64_t first, uint64_t count, cudaStream_t stream)
{
    DeviceInfo dev;
    srng_status st = current_device(&dev);
    if (st) return st;
    const int nbits = bit_length(s->stream_base + first + count - 1);
    const JumpTable &tab = jump_table(spacing_shift(s->spacing), 1);
    SRNG_CUDA_TRY(launch_mrg_place(s->d_state, s->n_streams, first, count, s->stream_base, s->y0, tab, nbits, stream,
                                   dev));
    return SRNG_OK;
}

// ------------------------------------------------------------ TinyMT32 sets
constexpr uint64_t kTmtMaxParams = 1ull << 20;

// The device polynomial table of set s under `key`, built on the host by
// `build` on first use and kept until srng_destroy (a launch in flight on any
// stream may still read an older table).
static srng_status tmt_table(srng_set *s, const std::array<uint64_t, 6> &key,
                             const std::function<void(std::vector<uint4> &)> &build, const uint4 **out)
{
    std::lock_guard<std::mutex> lk(s->tmt_mu);
    auto it = s->tmt_tables.find(key);
    if (it != s->tmt_tables.end()) {
        *out = it->second;
        return SRNG_OK;
    }
    if (s->tmt_tables.size() >= 64) {  // bound the cache: drop it once the device is idle
        SRNG_CUDA_TRY(cudaDeviceSynchronize());
        for (auto &kv : s->tmt_tables) cudaFree(kv.second);
        s->tmt_tables.clear();
    }
    std::vector<uint4> h;
    try { build(h); } catch (...) { return fail(SRNG_ERR_OOM, "host allocation failed"); }
    uint4 *d = nullptr;
    SRNG_CUDA_TRY(cudaMalloc(&d, std::max<size_t>(1, h.size()) * sizeof(uint4)));
    const cudaError_t e = cudaMemcpy(d, h.data(), h.size() * sizeof(uint4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "cudaMemcpy(TinyMT32 table)");
    }
    s->tmt_tables.emplace(key, d);
    *out = d;
    return SRNG_OK;
}

// x^(e_hi 2^64 + e_lo) mod p_g for the groups [g0, g0 + ng) (table kind `kind`).
static srng_status tmt_poly_table(srng_set *s, uint64_t kind, uint64_t e_hi, uint64_t e_lo, uint64_t g0,
                                  uint64_t ng, const uint4 **out)
{
    return tmt_table(s, {kind, e_hi, e_lo, g0, ng, 0},
                     [&](std::vector<uint4> &h) {
                         h.resize(ng);
                         for (uint64_t g = 0; g < ng; ++g) h[g] = poly_words(tmt_xpow(s->tmt_poly[g0 + g], e_hi, e_lo));
                     },
                     out);
}

// (x^(base))^(2^k) mod p_g, k < nbits, for the groups [g0, g0 + ng): the
// jump tables of chunk starts (base = chunk) and stream placement (2^64).
static srng_status tmt_pow2_table(srng_set *s, uint64_t kind, uint64_t e_hi, uint64_t e_lo, uint64_t g0,
                                  uint64_t ng, int nbits, const uint4 **out)
{
    return tmt_table(s, {kind, e_hi, e_lo, g0, ng, (uint64_t)nbits},
                     [&](std::vector<uint4> &h) {
                         h.resize(ng * nbits);
                         for (uint64_t g = 0; g < ng; ++g) {
                             const u128 p = s->tmt_poly[g0 + g];
                             u128 r = tmt_xpow(p, e_hi, e_lo);
                             for (int k = 0; k < nbits; ++k) {
                                 h[g * nbits + k] = poly_words(r);
                                 r = tmt_square_mod(p, r);
                             }
                         }
                     },
                     out);
}

// Every stream to its start: T^(j 2^64) of its group's seed state.
static srng_status tmt_place(srng_set *s, cudaStream_t stream)
{
    DeviceInfo dev;
    srng_status st = current_device(&dev);
    if (st) return st;
    const uint64_t ng = s->tmt_n_groups, gs = s->tmt_group_size;
    const int nbits = bit_length(std::min(gs, s->n_streams) - 1);
    const uint4 *seeds = nullptr, *jt = nullptr;
    st = tmt_table(s, {1, 0, 0, 0, ng, 0},
                   [&](std::vector<uint4> &h) {
                       h.resize(ng);
                       for (uint64_t g = 0; g < ng; ++g) {
                           uint32_t w[4];
                           const uint32_t *p = &s->tmt_params[3 * g];
                           tmt_seed_state(s->tmt_seed32, p[0], p[1], p[2], w);
                           h[g] = make_uint4(w[0], w[1], w[2], w[3]);
                       }
                   },
                   &seeds);
    if (st) return st;
    if (nbits > 0 && (st = tmt_pow2_table(s, 2, 1, 0, 0, ng, nbits, &jt))) return st;
    SRNG_CUDA_TRY(launch_tmt_place(s->d_tstate, s->n_streams, s->d_tparams, gs, seeds, jt, nbits, stream, dev));
    return SRNG_OK;
}

static void free_set(srng_set *s)
{
    if (s->d_state) cudaFree(s->d_state);
    if (s->d_start) cudaFree(s->d_start);
    if (s->d_pos) cudaFree(s->d_pos);
    if (s->d_tstate) cudaFree(s->d_tstate);
    if (s->d_tparams) cudaFree(s->d_tparams);
    for (auto &kv : s->tmt_tables) cudaFree(kv.second);
    delete s;
}

// polys: the parameter sets' characteristic polynomials when already known.
static srng_status tmt_create(srng_set **out, const uint32_t *params, const std::vector<u128> *polys,
                              uint64_t n_params, uint64_t group_size, uint64_t n_streams, uint64_t seed,
                              cudaStream_t stream)
{
    srng_set *s = new (std::nothrow) srng_set();
    if (!s) return fail(SRNG_ERR_OOM, "host allocation failed");
    s->gen = SRNG_TINYMT32;
    s->keyed = s->threefry = s->threefry64 = false;
    s->spacing = SRNG_SPACING_STREAM;
    s->n_streams = n_streams;
    s->stream_base = 0;
    s->seed = seed;
    s->key0 = (uint32_t)seed;
    s->key1 = (uint32_t)(seed >> 32);
    memset(s->y0, 0, sizeof s->y0);
    s->d_state = nullptr;
    s->d_start = nullptr;
    s->start_bytes = 0;
    s->d_pos = nullptr;
    s->max_pos = 0;
    s->d_stage[0] = s->d_stage[1] = nullptr;
    s->stage_bytes = 0;
    s->copy_stream = nullptr;
    s->tmt_group_size = group_size;
    s->tmt_n_groups = n_params;
    s->tmt_seed32 = (uint32_t)seed;
    cudaGetDevice(&s->device);
    srng_status st = SRNG_OK;
    try {
        s->tmt_params.assign(params, params + 3 * n_params);
        s->tmt_poly.resize(n_params);
    } catch (...) {
        free_set(s);
        return fail(SRNG_ERR_OOM, "host allocation failed");
    }
    for (uint64_t g = 0; g < n_params; ++g) {
        if (polys) {
            s->tmt_poly[g] = (*polys)[g];
        } else if (!tmt_max_period(params[3 * g], params[3 * g + 1], &s->tmt_poly[g])) {
            free_set(s);
            return fail(SRNG_ERR_ARG, "parameter set " + std::to_string(g) + " does not have period 2^127 - 1");
        }
    }
    std::vector<uint4> hp(n_params);
    for (uint64_t g = 0; g < n_params; ++g) hp[g] = make_uint4(params[3 * g], params[3 * g + 1], params[3 * g + 2], 0);
    s->start_bytes = 4 * n_streams * sizeof(uint32_t);
    cudaError_t e = cudaMalloc(&s->d_tstate, s->start_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_start, s->start_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_tparams, n_params * sizeof(uint4));
    if (e == cudaSuccess) e = cudaMemcpy(s->d_tparams, hp.data(), n_params * sizeof(uint4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_set(s);
        return cuda_fail(e, "TinyMT32 set allocation");
    }
    if ((st = tmt_place(s, stream))) {
        free_set(s);
        return st;
    }
    if ((e = cudaMemcpyAsync(s->d_start, s->d_tstate, s->start_bytes, cudaMemcpyDeviceToDevice, stream)) !=
        cudaSuccess) {
        free_set(s);
        return cuda_fail(e, "cudaMemcpyAsync(start states)");
    }
    if ((e = cudaStreamSynchronize(stream)) != cudaSuccess) {
        free_set(s);
        return cuda_fail(e, "cudaStreamSynchronize(create)");
    }
    *out = s;
    return SRNG_OK;
}

static srng_status create_common(srng_set **out, srng_gen gen, uint64_t seed, const uint32_t *state,
                                 uint64_t stream_base, uint64_t n_streams, srng_spacing spacing, void *cuda_stream)
{
    if (!out) return fail(SRNG_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!valid_gen(gen)) return fail(SRNG_ERR_ARG, "unknown generator");
    if (spacing != SRNG_SPACING_STREAM && spacing != SRNG_SPACING_SUBSTREAM)
        return fail(SRNG_ERR_ARG, "unknown spacing");
    if (n_streams == 0 || n_streams > (1ull << 40)) return fail(SRNG_ERR_ARG, "n_streams must be in [1, 2^40]");
    if (stream_base > UINT64_MAX - (n_streams - 1)) return fail(SRNG_ERR_RANGE, "stream numbers would pass 2^64 - 1");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    if (gen == SRNG_TINYMT32) {
        if (stream_base || state) return fail(SRNG_ERR_UNSUPPORTED, "TinyMT32 sets start at stream 0 from a seed");
        const uint64_t gs = 256, ng = (n_streams + gs - 1) / gs;
        if (ng > kTmtMaxParams) return fail(SRNG_ERR_ARG, "TinyMT32: at most 2^20 parameter sets (2^28 streams)");
        std::vector<uint32_t> prm;
        std::vector<u128> polys;
        try {
            prm.resize(3 * ng);
            polys.resize(ng);
        } catch (...) {
            return fail(SRNG_ERR_OOM, "host allocation failed");
        }
        tmt_find_params(seed, (uint32_t)ng, prm.data(), polys.data());
        return tmt_create(out, prm.data(), &polys, ng, gs, n_streams, seed, stream);
    }
    srng_set *s = new (std::nothrow) srng_set();
    if (!s) return fail(SRNG_ERR_OOM, "host allocation failed");
    s->keyed = gen == SRNG_PHILOX4X32_10_KEYED || gen == SRNG_THREEFRY4X32_20 || gen == SRNG_THREEFRY4X64_20;
    s->threefry = gen == SRNG_THREEFRY4X32_20 || gen == SRNG_THREEFRY4X64_20;
    s->threefry64 = gen == SRNG_THREEFRY4X64_20;
    s->gen = (srng_gen)kernel_gen(gen);
    s->spacing = spacing;
    s->n_streams = n_streams;
    s->stream_base = stream_base;
    s->seed = seed;
    s->d_state = nullptr;
    s->d_start = nullptr;
    s->start_bytes = 0;
    s->d_pos = nullptr;
    s->max_pos = 0;
    s->d_stage[0] = s->d_stage[1] = nullptr;
    s->stage_bytes = 0;
    s->copy_stream = nullptr;
    memset(s->y0, 0, sizeof s->y0);
    cudaGetDevice(&s->device);
    srng_status st = SRNG_OK;
    cudaError_t e;
    if (gen == SRNG_MRG32K3A) {
        if (state) memcpy(s->y0, state, sizeof s->y0);
        else seed_expand(seed, s->y0);
        s->start_bytes = 6 * n_streams * sizeof(uint32_t);
        e = cudaMalloc(&s->d_state, s->start_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_start, s->start_bytes);
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaMalloc(stream states)"); goto bad; }
        st = place_streams(s, 0, n_streams, stream);
        if (st) goto bad;
        e = cudaMemcpyAsync(s->d_start, s->d_state, s->start_bytes, cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaMemcpyAsync(start states)"); goto bad; }
    } else {
        s->key0 = (uint32_t)seed;
        s->key1 = (uint32_t)(seed >> 32);
        e = cudaMalloc(&s->d_pos, n_streams * sizeof(uint64_t));
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaMalloc(positions)"); goto bad; }
        e = cudaMemsetAsync(s->d_pos, 0, n_streams * sizeof(uint64_t), stream);
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaMemsetAsync(positions)"); goto bad; }
    }
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) { st = cuda_fail(e, "cudaStreamSynchronize(create)"); goto bad; }
    *out = s;
    return SRNG_OK;
bad:
    if (s->d_state) cudaFree(s->d_state);
    if (s->d_start) cudaFree(s->d_start);
    if (s->d_pos) cudaFree(s->d_pos);
    delete s;
    return st;
}

static srng_status check_range(const srng_set *s, uint64_t begin, uint64_t count)
{
    if (!s) return fail(SRNG_ERR_ARG, "set is NULL");
    if (begin > s->n_streams || count > s->n_streams - begin)
        return fail(SRNG_ERR_RANGE, "stream range [" + std::to_string(begin) + ", +" + std::to_string(count) +
                                        ") outside the set of " + std::to_string(s->n_streams));
    return SRNG_OK;
}

// Generation into a device buffer (shared by srng_generate* and the host path).
static srng_status generate_dev(srng_set *s, uint64_t b, uint64_t c, uint64_t n, srng_out type, void *out,
                                const srng_tune &t, cudaStream_t stream, const DeviceInfo &dev)
{
    if (s->gen == SRNG_MRG32K3A) {
        MrgGenArgs a;
        a.state = s->d_state;
        a.n_streams = s->n_streams;
        a.s_begin = b;
        a.s_count = c;
        a.n = n;
        uint64_t chunk = t.chunk;
        if (!chunk) {
            // enough items for about four waves of resident threads; when the
            // streams alone fill three quarters of a wave, one item per stream
            // (the kernels without jump code)
            const uint64_t resident = (uint64_t)dev.sm_count * t.blocks_per_sm * t.block_threads;
            const uint64_t want = 4 * resident;
            const uint64_t splits = 4 * c >= 3 * resident || c >= want ? 1 : (want + c - 1) / c;
            chunk = (n + splits - 1) / splits;
            chunk = ((chunk + 31) / 32) * 32;
            // a floor of 64 draws: a few long streams (64 x 2^16 FP64 draws)
            // then run as 65,536 items with radix-32 chunk starts
            if (chunk < 64) chunk = 64;
            // prefer a chunk that divides n (whole-row items, the fast kernel)
            for (uint64_t d = chunk; d <= 2 * chunk && d <= n; d += 32)
                if (n % d == 0) { chunk = d; break; }
        }
        if (chunk > n) chunk = n;
        a.chunk = chunk;
        a.cps = (n + chunk - 1) / chunk;
        a.nbits = bit_length(a.cps - 1);
        a.out = out;
        const JumpTable &tab = jump_table(0, chunk);
        const RadixTable *rt = a.cps >= 32 && a.cps % 32 == 0 ? &radix_table(chunk) : nullptr;
        srng_tune tt = t;
        if (!tt.vector_store) tt.vector_store = rt ? 3 : 1;
        SRNG_CUDA_TRY(launch_mrg_generate(a, type, tab, tt, stream, dev, rt));
        SRNG_CUDA_TRY(launch_mrg_apply(s->d_state, s->n_streams, b, c, mat_pow_shifted(0, n, 0), stream, dev, true));
    } else if (s->gen == SRNG_TINYMT32) {
        const uint64_t gs = s->tmt_group_size;
        TmtGenArgs a;
        a.state = s->d_tstate;
        a.n_streams = s->n_streams;
        a.params = s->d_tparams;
        a.group_size = gs;
        a.s_begin = b;
        a.s_count = c;
        a.n = n;
        a.out = out;
        uint64_t chunk = t.chunk;
        if (!chunk) {
            // about four waves of resident threads; a chunk start costs ~2,000
            // instructions per set bit of its index, so chunks stay >= 2048 draws
            // (measured at 2^18 streams x 4096: two chunks per stream beat one,
            // whose 2^18 items fill 1.1 waves of this kernel's resident threads)
            const uint64_t resident = (uint64_t)dev.sm_count * (t.blocks_per_sm ? t.blocks_per_sm : 8) * 256;
            const uint64_t want = 4 * resident;
            const uint64_t splits = c >= want ? 1 : (want + c - 1) / c;
            chunk = (n + splits - 1) / splits;
            chunk = std::max<uint64_t>(2048, ((chunk + 31) / 32) * 32);
        }
        if (chunk > n) chunk = n;
        a.chunk = chunk;
        a.cps = (n + chunk - 1) / chunk;
        a.nbits = bit_length(a.cps - 1);
        a.write_back = a.cps == 1 ? 1 : 0;
        const uint64_t g0 = b / gs, ng = (b + c - 1) / gs - g0 + 1;
        a.g0 = g0;
        a.jtab = nullptr;
        srng_status st;
        if (a.nbits > 0 && (st = tmt_pow2_table(s, 3, 0, chunk, g0, ng, a.nbits, &a.jtab))) return st;
        SRNG_CUDA_TRY(launch_tmt_generate(a, type, t, stream, dev));
        if (!a.write_back) {  // advance every stream by n (the chunks read the start state)
            const uint4 *adv = nullptr;
            if ((st = tmt_poly_table(s, 4, 0, n, g0, ng, &adv))) return st;
            SRNG_CUDA_TRY(launch_tmt_apply(s->d_tstate, s->n_streams, s->d_tparams, gs, b, c, adv, g0, stream, dev));
        }
    } else {
        PhiloxGenArgs a;
        a.stream_base = s->stream_base;
        a.k0 = s->key0;
        a.k1 = s->key1;
        a.keyed = s->keyed ? 1 : 0;
        a.threefry = s->threefry64 ? 2 : s->threefry ? 1 : 0;
        a.pos = s->d_pos;
        a.s_begin = b;
        a.s_count = c;
        a.n = n;
        a.out = out;
        SRNG_CUDA_TRY(launch_philox_generate(a, type, t, stream, dev));
        SRNG_CUDA_TRY(launch_philox_advance(s->d_pos, b, c, n, stream, dev));
        s->max_pos += n;
    }
    return SRNG_OK;
}

static srng_status generate_checks(srng_set *s, uint64_t b, uint64_t c, uint64_t n, srng_out type,
                                   const void *out)
{
    srng_status st = check_range(s, b, c);
    if (st) return st;
    if (!valid_gen_out(type)) return fail(SRNG_ERR_ARG, "unknown output type");
    if (type == SRNG_OUT_NORMAL_F32 && (n & 1) && (s->gen == SRNG_MRG32K3A || s->gen == SRNG_TINYMT32))
        return fail(SRNG_ERR_ARG, "normal output of a state-based generator takes draws in pairs: n must be even");
    if (c == 0 || n == 0) return SRNG_OK;
    if (!out) return fail(SRNG_ERR_ARG, "output pointer is NULL");
    if (reinterpret_cast<uintptr_t>(out) % out_size(type))
        return fail(SRNG_ERR_ARG, "output pointer not aligned to the element size");
    if (n > (1ull << 62) || c > (1ull << 62) / n || c * n > (1ull << 62) / out_size(type))
        return fail(SRNG_ERR_ARG, "output size overflows");
    if (s->gen == SRNG_PHILOX4X32_10 && n > UINT64_MAX - s->max_pos)
        return fail(SRNG_ERR_RANGE, "a Philox position would pass 2^64 - 1");
    return SRNG_OK;
}

}  // namespace srng_impl

using namespace srng_impl;

extern "C" {

const char *srng_last_error(void) { return t_last_error.c_str(); }

const char *srng_status_string(srng_status status)
{
    switch (status) {
    case SRNG_OK: return "SRNG_OK";
    case SRNG_ERR_ARG: return "SRNG_ERR_ARG";
    case SRNG_ERR_OOM: return "SRNG_ERR_OOM";
    case SRNG_ERR_STATE: return "SRNG_ERR_STATE";
    case SRNG_ERR_CUDA: return "SRNG_ERR_CUDA";
    case SRNG_ERR_BUDGET: return "SRNG_ERR_BUDGET";
    case SRNG_ERR_TIMEOUT: return "SRNG_ERR_TIMEOUT";
    case SRNG_ERR_RANGE: return "SRNG_ERR_RANGE";
    case SRNG_ERR_CLOSED: return "SRNG_ERR_CLOSED";
    case SRNG_ERR_UNSUPPORTED: return "SRNG_ERR_UNSUPPORTED";
    }
    return "SRNG_UNKNOWN_STATUS";
}

int srng_abi_version(void) { return SRNG_ABI_VERSION; }

srng_status srng_create(srng_set **out, srng_gen gen, uint64_t seed, uint64_t n_streams, srng_spacing spacing,
                        void *cuda_stream)
{
    clear_error();
    return create_common(out, gen, seed, nullptr, 0, n_streams, spacing, cuda_stream);
}

srng_status srng_create_range(srng_set **out, srng_gen gen, uint64_t seed, const uint32_t state[6],
                              uint64_t stream_base, uint64_t n_streams, srng_spacing spacing, void *cuda_stream)
{
    clear_error();
    if (state) {
        if (gen != SRNG_MRG32K3A) return fail(SRNG_ERR_ARG, "an explicit seed state is MRG32k3a only");
        if (!state_valid(state))
            return fail(SRNG_ERR_STATE, "seed state must have x1 words < m1, x2 words < m2, no all-zero component");
    }
    return create_common(out, gen, seed, state, stream_base, n_streams, spacing, cuda_stream);
}

srng_status srng_create_from_state(srng_set **out, const uint32_t state[6], uint64_t n_streams,
                                   srng_spacing spacing, void *cuda_stream)
{
    clear_error();
    if (!state) return fail(SRNG_ERR_ARG, "state is NULL");
    if (!state_valid(state))
        return fail(SRNG_ERR_STATE, "seed state must have x1 words < m1, x2 words < m2, no all-zero component");
    return create_common(out, SRNG_MRG32K3A, 0, state, 0, n_streams, spacing, cuda_stream);
}

srng_status srng_create_tinymt(srng_set **out, const uint32_t *params, uint64_t n_params, uint64_t group_size,
                               uint64_t seed, void *cuda_stream)
{
    clear_error();
    if (!out || !params) return fail(SRNG_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (n_params == 0 || n_params > kTmtMaxParams) return fail(SRNG_ERR_ARG, "n_params must be in [1, 2^20]");
    if (group_size == 0 || group_size > (1ull << 40) / n_params)
        return fail(SRNG_ERR_ARG, "group_size must be >= 1 and n_params * group_size <= 2^40");
    return tmt_create(out, params, nullptr, n_params, group_size, n_params * group_size, seed,
                      static_cast<cudaStream_t>(cuda_stream));
}

srng_status srng_tinymt_find_params(uint64_t seed, uint32_t count, uint32_t *params_out)
{
    clear_error();
    if (count && !params_out) return fail(SRNG_ERR_ARG, "params_out is NULL");
    if (count > kTmtMaxParams) return fail(SRNG_ERR_ARG, "at most 2^20 parameter sets per call");
    tmt_find_params(seed, count, params_out, nullptr);
    return SRNG_OK;
}

srng_status srng_tinymt_check_params(uint32_t mat1, uint32_t mat2, int *max_period)
{
    clear_error();
    if (!max_period) return fail(SRNG_ERR_ARG, "max_period is NULL");
    *max_period = tmt_max_period(mat1, mat2, nullptr) ? 1 : 0;
    return SRNG_OK;
}

srng_status srng_destroy(srng_set *set)
{
    clear_error();
    if (!set) return SRNG_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(set->device);
    cudaDeviceSynchronize();
    if (set->d_state) cudaFree(set->d_state);
    if (set->d_pos) cudaFree(set->d_pos);
    if (set->d_tstate) cudaFree(set->d_tstate);
    if (set->d_tparams) cudaFree(set->d_tparams);
    for (auto &kv : set->tmt_tables) cudaFree(kv.second);
    for (int i = 0; i < 2; ++i) {
        if (set->d_stage[i]) cudaFree(set->d_stage[i]);
    }
    if (set->copy_stream) {
        cudaStreamDestroy(set->copy_stream);
        for (int i = 0; i < 2; ++i) {
            cudaEventDestroy(set->ev_gen[i]);
            cudaEventDestroy(set->ev_copy[i]);
        }
    }
    cudaSetDevice(prev);
    delete set;
    return SRNG_OK;
}

srng_status srng_reset(srng_set *set, void *cuda_stream)
{
    clear_error();
    if (!set) return fail(SRNG_ERR_ARG, "set is NULL");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    if (set->gen == SRNG_MRG32K3A || set->gen == SRNG_TINYMT32) {
        // the start states placed at creation, kept beside the working states
        SRNG_CUDA_TRY(cudaMemcpyAsync(set->gen == SRNG_MRG32K3A ? set->d_state : set->d_tstate, set->d_start,
                                      set->start_bytes, cudaMemcpyDeviceToDevice, stream));
        return SRNG_OK;
    }
    SRNG_CUDA_TRY(cudaMemsetAsync(set->d_pos, 0, set->n_streams * sizeof(uint64_t), stream));
    set->max_pos = 0;
    return SRNG_OK;
}

srng_status srng_describe(const srng_set *set, srng_set_desc *out)
{
    clear_error();
    if (!set || !out) return fail(SRNG_ERR_ARG, "NULL argument");
    memset(out, 0, sizeof *out);
    out->gen = set->threefry ? (srng_gen)inst_gen(set) : set->keyed ? SRNG_PHILOX4X32_10_KEYED : set->gen;  // TinyMT32 too
    out->spacing = set->spacing;
    out->n_streams = set->n_streams;
    out->seed = set->seed;
    if (set->gen == SRNG_MRG32K3A) memcpy(out->seed_state, set->y0, sizeof set->y0);
    else { out->seed_state[0] = set->key0; out->seed_state[1] = set->key1; }
    out->stream_base = set->stream_base;
    return SRNG_OK;
}

srng_status srng_get_device_view(const srng_set *set, srng_dev_view *out)
{
    clear_error();
    if (!set || !out) return fail(SRNG_ERR_ARG, "NULL argument");
    memset(out, 0, sizeof *out);
    out->gen = (int32_t)inst_gen(set);
    out->key0 = set->key0;
    out->key1 = set->key1;
    out->flags = set->keyed && !set->threefry ? 1u : 0u;
    out->tinymt_state = set->d_tstate;
    out->tinymt_params = reinterpret_cast<const uint32_t *>(set->d_tparams);
    out->tinymt_group_size = set->tmt_group_size;
    out->n_streams = set->n_streams;
    out->mrg_state = set->d_state;
    out->philox_pos = set->d_pos;
    out->stream_base = set->stream_base;
    return SRNG_OK;
}

srng_status srng_jump(srng_set *set, uint64_t stream_begin, uint64_t count, srng_jump_unit unit, uint64_t n_hi,
                      uint64_t n_lo, void *cuda_stream)
{
    clear_error();
    srng_status st = check_range(set, stream_begin, count);
    if (st) return st;
    if (unit != SRNG_JUMP_DRAWS && unit != SRNG_JUMP_SUBSTREAMS && unit != SRNG_JUMP_STREAMS)
        return fail(SRNG_ERR_ARG, "unknown jump unit");
    if (count == 0) return SRNG_OK;
    DeviceInfo dev;
    if ((st = current_device(&dev))) return st;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    if (set->gen == SRNG_MRG32K3A) {
        const int shift = unit == SRNG_JUMP_DRAWS ? 0 : unit == SRNG_JUMP_SUBSTREAMS ? 76 : 127;
        SRNG_CUDA_TRY(launch_mrg_apply(set->d_state, set->n_streams, stream_begin, count,
                                       mat_pow_shifted(n_hi, n_lo, shift), stream, dev));
        return SRNG_OK;
    }
    if (set->gen == SRNG_TINYMT32) {
        if (unit != SRNG_JUMP_DRAWS) return fail(SRNG_ERR_UNSUPPORTED, "TinyMT32 streams jump by draws only");
        const uint64_t gs = set->tmt_group_size, g0 = stream_begin / gs, ng = (stream_begin + count - 1) / gs - g0 + 1;
        const uint4 *poly = nullptr;
        if ((st = tmt_poly_table(set, 5, n_hi, n_lo, g0, ng, &poly))) return st;
        SRNG_CUDA_TRY(launch_tmt_apply(set->d_tstate, set->n_streams, set->d_tparams, gs, stream_begin, count, poly, g0,
                                       stream, dev));
        return SRNG_OK;
    }
    if (unit != SRNG_JUMP_DRAWS) return fail(SRNG_ERR_UNSUPPORTED, "Philox streams jump by draws only");
    if (n_hi || n_lo > UINT64_MAX - set->max_pos) return fail(SRNG_ERR_RANGE, "a Philox position would pass 2^64 - 1");
    SRNG_CUDA_TRY(launch_philox_advance(set->d_pos, stream_begin, count, n_lo, stream, dev));
    set->max_pos += n_lo;
    return SRNG_OK;
}

srng_status srng_generate_tuned(srng_set *set, uint64_t stream_begin, uint64_t stream_count, uint64_t n_per_stream,
                                srng_out type, void *out_dev, const srng_tune *tune, void *cuda_stream)
{
    clear_error();
    srng_status st = generate_checks(set, stream_begin, stream_count, n_per_stream, type, out_dev);
    if (st) return st;
    if ((st = check_tune(tune))) return st;
    if (stream_count == 0 || n_per_stream == 0) return SRNG_OK;
    DeviceInfo dev;
    if ((st = current_device(&dev))) return st;
    const srng_tune t = effective_tune(set->gen, type, tune);
    return generate_dev(set, stream_begin, stream_count, n_per_stream, type, out_dev, t,
                        static_cast<cudaStream_t>(cuda_stream), dev);
}

srng_status srng_generate(srng_set *set, uint64_t stream_begin, uint64_t stream_count, uint64_t n_per_stream,
                          srng_out type, void *out_dev, void *cuda_stream)
{
    return srng_generate_tuned(set, stream_begin, stream_count, n_per_stream, type, out_dev, nullptr, cuda_stream);
}

srng_status srng_generate_host(srng_set *set, uint64_t stream_begin, uint64_t stream_count, uint64_t n_per_stream,
                               srng_out type, void *out_host, void *cuda_stream)
{
    clear_error();
    srng_status st = generate_checks(set, stream_begin, stream_count, n_per_stream, type, out_host);
    if (st) return st;
    if (stream_count == 0 || n_per_stream == 0) return SRNG_OK;
    DeviceInfo dev;
    if ((st = current_device(&dev))) return st;
    std::lock_guard<std::mutex> lk(set->mu);
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    {
        // Pinned host memory the device can address (cudaHostAlloc /
        // cudaHostRegister): the kernels store straight into it over the
        // host link, no staging and no copy engine.
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, out_host) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
            attr.devicePointer) {
            srng_tune t = effective_tune(set->gen, type, nullptr);
            // whole 128-byte lines per warp store (staged rows) cross the host
            // link best; per-lane 32-byte row pieces measured 20% slower there
            t.vector_store = 1;
            st = generate_dev(set, stream_begin, stream_count, n_per_stream, type, attr.devicePointer, t, stream, dev);
            if (st) return st;
            SRNG_CUDA_TRY(cudaStreamSynchronize(stream));
            return SRNG_OK;
        }
        cudaGetLastError();  // clear a "not a device pointer" result for pageable memory
    }
    const size_t kStage = 256ull << 20;
    if (!set->d_stage[0]) {
        for (int i = 0; i < 2; ++i) SRNG_CUDA_TRY(cudaMalloc(&set->d_stage[i], kStage));
        SRNG_CUDA_TRY(cudaStreamCreateWithFlags(&set->copy_stream, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            SRNG_CUDA_TRY(cudaEventCreateWithFlags(&set->ev_gen[i], cudaEventDisableTiming));
            SRNG_CUDA_TRY(cudaEventCreateWithFlags(&set->ev_copy[i], cudaEventDisableTiming));
        }
        set->stage_bytes = kStage;
    }
    const srng_tune t = effective_tune(set->gen, type, nullptr);
    const size_t esz = out_size(type);
    const uint64_t stage_elems = set->stage_bytes / esz;
    // Pieces: whole streams when a stream fits the stage, else consecutive
    // parts of one stream (generation of part k moves the stream to part k+1).
    struct Piece { uint64_t s, cnt, n, host_off; };
    std::vector<Piece> pieces;
    if (n_per_stream <= stage_elems) {
        const uint64_t per = stage_elems / n_per_stream;
        for (uint64_t s = 0; s < stream_count; s += per) {
            const uint64_t cnt = std::min(per, stream_count - s);
            pieces.push_back({stream_begin + s, cnt, n_per_stream, s * n_per_stream});
        }
    } else {
        for (uint64_t s = 0; s < stream_count; ++s)
            for (uint64_t k = 0; k < n_per_stream; k += stage_elems)
                pieces.push_back({stream_begin + s, 1, std::min(stage_elems, n_per_stream - k), s * n_per_stream + k});
    }
    bool used[2] = {false, false};
    for (size_t i = 0; i < pieces.size(); ++i) {
        const int slot = (int)(i & 1);
        const Piece &p = pieces[i];
        if (used[slot]) SRNG_CUDA_TRY(cudaStreamWaitEvent(stream, set->ev_copy[slot], 0));
        st = generate_dev(set, p.s, p.cnt, p.n, type, set->d_stage[slot], t, stream, dev);
        if (st) return st;
        SRNG_CUDA_TRY(cudaEventRecord(set->ev_gen[slot], stream));
        SRNG_CUDA_TRY(cudaStreamWaitEvent(set->copy_stream, set->ev_gen[slot], 0));
        SRNG_CUDA_TRY(cudaMemcpyAsync(static_cast<char *>(out_host) + p.host_off * esz, set->d_stage[slot],
                                      p.cnt * p.n * esz, cudaMemcpyDeviceToHost, set->copy_stream));
        SRNG_CUDA_TRY(cudaEventRecord(set->ev_copy[slot], set->copy_stream));
        used[slot] = true;
    }
    SRNG_CUDA_TRY(cudaStreamSynchronize(set->copy_stream));
    SRNG_CUDA_TRY(cudaStreamSynchronize(stream));
    return SRNG_OK;
}

srng_status srng_get_state(const srng_set *set, uint64_t stream_begin, uint64_t count, void *state_host,
                           void *cuda_stream)
{
    clear_error();
    srng_status st = check_range(set, stream_begin, count);
    if (st) return st;
    if (count == 0) return SRNG_OK;
    if (!state_host) return fail(SRNG_ERR_ARG, "state_host is NULL");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    if (set->gen == SRNG_TINYMT32) {
        std::vector<uint32_t> soa;
        try { soa.resize(4 * count); } catch (...) { return fail(SRNG_ERR_OOM, "host allocation failed"); }
        SRNG_CUDA_TRY(cudaMemcpy2DAsync(soa.data(), count * sizeof(uint32_t), set->d_tstate + stream_begin,
                                        set->n_streams * sizeof(uint32_t), count * sizeof(uint32_t), 4,
                                        cudaMemcpyDeviceToHost, stream));
        SRNG_CUDA_TRY(cudaStreamSynchronize(stream));
        uint32_t *h = static_cast<uint32_t *>(state_host);
        for (uint64_t i = 0; i < count; ++i)
            for (int j = 0; j < 4; ++j) h[4 * i + j] = soa[j * count + i];
        return SRNG_OK;
    }
    if (set->gen == SRNG_PHILOX4X32_10) {
        SRNG_CUDA_TRY(cudaMemcpyAsync(state_host, set->d_pos + stream_begin, count * sizeof(uint64_t),
                                      cudaMemcpyDeviceToHost, stream));
        SRNG_CUDA_TRY(cudaStreamSynchronize(stream));
        return SRNG_OK;
    }
    std::vector<uint32_t> soa;
    try { soa.resize(6 * count); } catch (...) { return fail(SRNG_ERR_OOM, "host allocation failed"); }
    SRNG_CUDA_TRY(cudaMemcpy2DAsync(soa.data(), count * sizeof(uint32_t), set->d_state + stream_begin,
                                    set->n_streams * sizeof(uint32_t), count * sizeof(uint32_t), 6,
                                    cudaMemcpyDeviceToHost, stream));
    SRNG_CUDA_TRY(cudaStreamSynchronize(stream));
    uint32_t *h = static_cast<uint32_t *>(state_host);
    for (uint64_t i = 0; i < count; ++i)
        for (int j = 0; j < 6; ++j) h[6 * i + j] = soa[j * count + i];
    return SRNG_OK;
}

srng_status srng_set_state(srng_set *set, uint64_t stream_begin, uint64_t count, const void *state_host,
                           void *cuda_stream)
{
    clear_error();
    srng_status st = check_range(set, stream_begin, count);
    if (st) return st;
    if (count == 0) return SRNG_OK;
    if (!state_host) return fail(SRNG_ERR_ARG, "state_host is NULL");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    if (set->gen == SRNG_TINYMT32) {
        const uint32_t *h = static_cast<const uint32_t *>(state_host);
        std::vector<uint32_t> soa;
        try { soa.resize(4 * count); } catch (...) { return fail(SRNG_ERR_OOM, "host allocation failed"); }
        for (uint64_t i = 0; i < count; ++i) {
            if ((h[4 * i] & 0x7fffffffu) == 0 && h[4 * i + 1] == 0 && h[4 * i + 2] == 0 && h[4 * i + 3] == 0)
                return fail(SRNG_ERR_STATE, "TinyMT32 state " + std::to_string(i) + " is all zero");
            for (int j = 0; j < 4; ++j) soa[j * count + i] = h[4 * i + j];
        }
        SRNG_CUDA_TRY(cudaMemcpy2DAsync(set->d_tstate + stream_begin, set->n_streams * sizeof(uint32_t), soa.data(),
                                        count * sizeof(uint32_t), count * sizeof(uint32_t), 4, cudaMemcpyHostToDevice,
                                        stream));
        SRNG_CUDA_TRY(cudaStreamSynchronize(stream));
        return SRNG_OK;
    }
    if (set->gen == SRNG_PHILOX4X32_10) {
        const uint64_t *p = static_cast<const uint64_t *>(state_host);
        uint64_t mx = 0;
        for (uint64_t i = 0; i < count; ++i) mx = std::max(mx, p[i]);
        SRNG_CUDA_TRY(cudaMemcpyAsync(set->d_pos + stream_begin, state_host, count * sizeof(uint64_t),
                                      cudaMemcpyHostToDevice, stream));
        SRNG_CUDA_TRY(cudaStreamSynchronize(stream));
        set->max_pos = std::max(set->max_pos, mx);
        return SRNG_OK;
    }
    const uint32_t *h = static_cast<const uint32_t *>(state_host);
    for (uint64_t i = 0; i < count; ++i)
        if (!state_valid(h + 6 * i))
            return fail(SRNG_ERR_STATE, "state of stream " + std::to_string(stream_begin + i) + " is invalid");
    std::vector<uint32_t> soa;
    try { soa.resize(6 * count); } catch (...) { return fail(SRNG_ERR_OOM, "host allocation failed"); }
    for (uint64_t i = 0; i < count; ++i)
        for (int j = 0; j < 6; ++j) soa[j * count + i] = h[6 * i + j];
    SRNG_CUDA_TRY(cudaMemcpy2DAsync(set->d_state + stream_begin, set->n_streams * sizeof(uint32_t), soa.data(),
                                    count * sizeof(uint32_t), count * sizeof(uint32_t), 6, cudaMemcpyHostToDevice,
                                    stream));
    SRNG_CUDA_TRY(cudaStreamSynchronize(stream));
    return SRNG_OK;
}

srng_status srng_set_tune(srng_gen gen, srng_out type, const srng_tune *tune)
{
    clear_error();
    if (!valid_gen(gen) || !valid_out(type)) return fail(SRNG_ERR_ARG, "unknown generator or output type");
    srng_status st = check_tune(tune);
    if (st) return st;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const int g = tune_row(kernel_gen(gen));
    if (tune) {
        g_tune[g][type] = *tune;
        g_tune_set[g][type] = true;
    } else {
        g_tune_set[g][type] = false;
    }
    return SRNG_OK;
}

srng_status srng_get_tune(srng_gen gen, srng_out type, srng_tune *out)
{
    clear_error();
    if (!valid_gen(gen) || !valid_out(type) || !out) return fail(SRNG_ERR_ARG, "bad argument");
    *out = effective_tune(gen, type, nullptr);
    return SRNG_OK;
}

srng_status srng_convert(srng_gen gen, srng_out type, const uint32_t *in_dev, uint64_t n, void *out_dev,
                         void *cuda_stream)
{
    clear_error();
    if (!valid_gen(gen) || !valid_out(type)) return fail(SRNG_ERR_ARG, "unknown generator or output type");
    if (n == 0) return SRNG_OK;
    if (!in_dev || !out_dev) return fail(SRNG_ERR_ARG, "NULL pointer");
    if (reinterpret_cast<uintptr_t>(in_dev) % 4 || reinterpret_cast<uintptr_t>(out_dev) % out_size(type))
        return fail(SRNG_ERR_ARG, "misaligned pointer");
    DeviceInfo dev;
    srng_status st = current_device(&dev);
    if (st) return st;
    SRNG_CUDA_TRY(launch_convert(gen, type, in_dev, n, out_dev, static_cast<cudaStream_t>(cuda_stream), dev));
    return SRNG_OK;
}

srng_status srng_transform(srng_dist dist, const float *in_dev, uint64_t n, float *out_dev, void *cuda_stream)
{
    clear_error();
    if (dist != SRNG_DIST_EXPONENTIAL && dist != SRNG_DIST_NORMAL) return fail(SRNG_ERR_ARG, "unknown distribution");
    if (n == 0) return SRNG_OK;
    if (!in_dev || !out_dev) return fail(SRNG_ERR_ARG, "NULL pointer");
    if (dist == SRNG_DIST_NORMAL && (n & 1)) return fail(SRNG_ERR_ARG, "normal variates come in pairs: n must be even");
    const uintptr_t align = dist == SRNG_DIST_NORMAL ? 8 : 4;
    if (reinterpret_cast<uintptr_t>(in_dev) % align || reinterpret_cast<uintptr_t>(out_dev) % align)
        return fail(SRNG_ERR_ARG, "misaligned pointer");
    DeviceInfo dev;
    srng_status st = current_device(&dev);
    if (st) return st;
    SRNG_CUDA_TRY(launch_transform(dist, in_dev, n, out_dev, static_cast<cudaStream_t>(cuda_stream), dev));
    return SRNG_OK;
}

srng_status srng_seed_expand(uint64_t seed, uint32_t state[6])
{
    clear_error();
    if (!state) return fail(SRNG_ERR_ARG, "state is NULL");
    seed_expand(seed, state);
    return SRNG_OK;
}

srng_status srng_jump_matrix(srng_jump_unit unit, uint64_t n_hi, uint64_t n_lo, uint32_t a1[9], uint32_t a2[9])
{
    clear_error();
    if (!a1 || !a2) return fail(SRNG_ERR_ARG, "NULL output");
    if (unit != SRNG_JUMP_DRAWS && unit != SRNG_JUMP_SUBSTREAMS && unit != SRNG_JUMP_STREAMS)
        return fail(SRNG_ERR_ARG, "unknown jump unit");
    const int shift = unit == SRNG_JUMP_DRAWS ? 0 : unit == SRNG_JUMP_SUBSTREAMS ? 76 : 127;
    MatPair m = mat_pow_shifted(n_hi, n_lo, shift);
    memcpy(a1, m.a, 9 * sizeof(uint32_t));
    memcpy(a2, m.a + 9, 9 * sizeof(uint32_t));
    return SRNG_OK;
}

}  // extern "C"
