// Scan and stable radix sort used by the ordering, pattern and schedule
// steps, plus error reporting.  Written for sm_103a; no library kernels.
#include <cstdio>
#include <cmath>
#include <atomic>
#include <mutex>

#include <vector>

#include "common.cuh"
#include "covariance.cuh"

namespace kc {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error_cstr() { return g_last_error.c_str(); }
kc_status fail(kc_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}
kc_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? KC_ENOMEM : KC_ECUDA;
}

static std::atomic<int64_t> g_launches{0};
static thread_local double g_factor_ms = 0.0;
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
void set_factor_kernel_ms(double ms) { g_factor_ms = ms; }
double factor_kernel_ms() { return g_factor_ms; }

// One private stream-ordered pool per device for the library's scratch.  The
// device's default pool (what cudaMallocAsync uses for everyone else in the
// process) is left as it is.  The private pool keeps up to SCRATCH_KEEP_BYTES
// of freed memory mapped between calls; kc_scratch_trim hands it back.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64] = {nullptr};

kc_status scratch_pool(cudaMemPool_t* out) {
    int dev = 0;
    KC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(KC_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        KC_CUDA(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = SCRATCH_KEEP_BYTES;
        cudaError_t e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return cuda_fail(e, "cudaMemPoolSetAttribute(scratch pool)");
        }
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return KC_OK;
}

kc_status scratch_alloc(void** p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool = nullptr;
    KC_TRY(scratch_pool(&pool));
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocFromPoolAsync(scratch)");
    return KC_OK;
}

kc_status scratch_trim(int64_t keep_bytes) {
    if (keep_bytes < 0) return fail(KC_EINVAL, "kc_scratch_trim: keep_bytes < 0");
    int dev = 0;
    KC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(KC_EINVAL, "device index out of range");
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        pool = g_pools[dev];
    }
    if (!pool) return KC_OK;  // nothing allocated on this device yet
    KC_CUDA(cudaMemPoolTrimTo(pool, (size_t)keep_bytes));
    return KC_OK;
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// Taylor coefficients of 1/Gamma(z) = sum_{k>=1} c_k z^k (Abramowitz & Stegun
// 6.1.34): 1/Gamma(1+mu) = sum_k c_k mu^{k-1}, entire, so for |mu| <= 1/2 the
// even and odd parts give Temme's gamma_1 and gamma_2 without the
// cancellation of their difference quotient.
static const double RGAMMA_TAYLOR[26] = {
    1.0, 0.5772156649015329, -0.6558780715202538, -0.0420026350340952, 0.1665386113822915,
    -0.0421977345555443, -0.0096219715278770, 0.0072189432466630, -0.0011651675918591,
    -0.0002152416741149, 0.0001280502823882, -0.0000201348547807, -0.0000012504934821,
    0.0000011330272320, -0.0000002056338417, 0.0000000061160950, 0.0000000050020075,
    -0.0000000011812746, 0.0000000001043427, 0.0000000000077823, -0.0000000000036968,
    0.0000000000005100, -0.0000000000000206, -0.0000000000000054, 0.0000000000000014,
    0.0000000000000001};

kc_status kernel_params(const kc_kernel* k, KernelParams* out) {
    if (!k) return fail(KC_EINVAL, "kernel parameters are NULL");
    if (!(k->ell > 0.0) || !(k->sigma2 > 0.0) || !(k->nugget >= 0.0))
        return fail(KC_EINVAL, "kernel needs ell > 0, sigma2 > 0, nugget >= 0");
    *out = KernelParams{};
    out->sigma2 = k->sigma2;
    out->nugget = k->nugget;
    if (k->family == KC_CAUCHY) {
        if (!(k->alpha > 0.0 && k->alpha <= 2.0) || !(k->beta > 0.0))
            return fail(KC_EINVAL, "the Cauchy class needs 0 < alpha <= 2 and beta > 0");
        out->nu_code = 4;
        out->scale = 1.0 / k->ell;
        out->alpha = k->alpha;
        out->expo = -k->beta / k->alpha;
        return KC_OK;
    }
    if (k->family != KC_MATERN) return fail(KC_EINVAL, "family must be KC_MATERN or KC_CAUCHY");
    if (!(k->nu > 0.0 && k->nu <= 50.0)) return fail(KC_EINVAL, "nu must be in (0, 50]");
    out->scale = sqrt(2.0 * k->nu) / k->ell;
    out->nu = k->nu;
    if (k->nu == 0.5) out->nu_code = 0;
    else if (k->nu == 1.5) out->nu_code = 1;
    else if (k->nu == 2.5) out->nu_code = 2;
    else {
        out->nu_code = 3;
        const double n = floor(k->nu + 0.5);
        const double mu = k->nu - n;
        double odd = 0.0, even = 0.0;  // sum c_{2m} mu^{2m-2}, sum c_{2m+1} mu^{2m}
        for (int i = 25; i >= 0; --i) {
            if (i & 1) odd = odd * mu * mu + RGAMMA_TAYLOR[i];
            else even = even * mu * mu + RGAMMA_TAYLOR[i];
        }
        out->n = (int)n;
        out->mu = mu;
        out->gam1 = -odd;
        out->gam2 = even;
        out->gp = 1.0 / (even + mu * odd);  // Gamma(1 + mu)
        out->gm = 1.0 / (even - mu * odd);  // Gamma(1 - mu)
        out->fact = mu == 0.0 ? 1.0 : mu * M_PI / sin(mu * M_PI);
        out->lognorm = (1.0 - k->nu) * log(2.0) - lgamma(k->nu);
        out->iser = fabs(mu) >= 0.02 ? 1 : 0;
        out->cheb = k->nu <= 8.0 ? 1 : 0;
    }
    return KC_OK;
}

void matern_coef_table(const KernelParams& kp, double* tab) {
    const double nu = kp.nu;
    // power series: a_0 = 1 (reflection formula), a_k = a_{k-1} / (k (k - nu));
    // b_0 = 4^{-nu} Gamma(1 - nu) / Gamma(1 + nu), b_k = b_{k-1} / (k (k + nu))
    double a = 1.0, b = kp.iser ? pow(4.0, -nu) * tgamma(1.0 - nu) / tgamma(1.0 + nu) : 0.0;
    for (int k = 0; k < KC_ISER; ++k) {
        if (k > 0) {
            a /= k * (k - nu);
            b /= k * (k + nu);
        }
        tab[k] = kp.iser ? a : 0.0;
        tab[KC_ISER + k] = b;
    }
    // Chebyshev interpolants of e^t sqrt(t) K_nu(t) on [2^{p+1}, 2^{p+2}]
    double f[KC_CHEB_N];
    for (int p = 0; p < KC_CHEB_P; ++p) {
        double* c = tab + 2 * KC_ISER + p * KC_CHEB_N;
        for (int j = 0; j < KC_CHEB_N; ++j) {
            const double t = ldexp(3.0 + cos(M_PI * (j + 0.5) / KC_CHEB_N), p);
            double g0, g1;
            steed_scaled(t, kp.mu, g0, g1);
            f[j] = k_upward(t, kp.mu, kp.n, g0, g1);
        }
        for (int k = 0; k < KC_CHEB_N; ++k) {
            double sum = 0.0;
            for (int j = 0; j < KC_CHEB_N; ++j) sum += f[j] * cos(M_PI * k * (j + 0.5) / KC_CHEB_N);
            c[k] = kp.cheb ? 2.0 * sum / KC_CHEB_N : 0.0;
        }
    }
}

kc_status upload_coef(KernelParams& kp, double* dst, cudaStream_t s) {
    if (kp.nu_code != 3) return KC_OK;
    std::vector<double> tab(KC_COEF_LEN);
    matern_coef_table(kp, tab.data());
    // from pageable memory the call returns once the table is staged, so it may
    // go out of scope afterwards
    KC_CUDA(cudaMemcpyAsync(dst, tab.data(), sizeof(double) * KC_COEF_LEN, cudaMemcpyHostToDevice, s));
    kp.coef = dst;
    return KC_OK;
}

kc_status upload_coef(KernelParams& kp, Arena& A, cudaStream_t s) {
    if (kp.nu_code != 3) return KC_OK;
    double* dst;
    KC_TRY(A.get(&dst, KC_COEF_LEN));
    return upload_coef(kp, dst, s);
}

// ------------------------------------------------------------------ scan
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename Tin>
__global__ void scan_reduce_k(const Tin* __restrict__ in, int64_t n, int64_t* __restrict__ bsum) {
    __shared__ int64_t red[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
    for (int it = 0; it < SCAN_ITEMS; ++it) {
        int64_t i = base + (int64_t)it * SCAN_THREADS + threadIdx.x;
        if (i < n) s += (int64_t)in[i];
    }
    s = warp_sum(s);
    if (lane_id() == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t v = threadIdx.x < SCAN_THREADS / 32 ? red[threadIdx.x] : 0;
        v = warp_sum(v);
        if (threadIdx.x == 0) bsum[blockIdx.x] = v;
    }
}

// Each block scans its tile (blocked arrangement) and adds its block offset.
template <typename Tin>
__global__ void scan_tile_k(const Tin* __restrict__ in, int64_t n, const int64_t* __restrict__ boff,
                            int64_t* __restrict__ out) {
    __shared__ int64_t wsum[SCAN_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t t = 0;
#pragma unroll
    for (int it = 0; it < SCAN_ITEMS; ++it) {
        int64_t i = base + it;
        v[it] = i < n ? (int64_t)in[i] : 0;
        t += v[it];
    }
    // inclusive warp scan of thread totals
    int lane = lane_id(), w = threadIdx.x >> 5;
    int64_t incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int64_t woff = 0;
    for (int q = 0; q < w; ++q) woff += wsum[q];
    int64_t run = boff[blockIdx.x] + woff + incl - t;
#pragma unroll
    for (int it = 0; it < SCAN_ITEMS; ++it) {
        int64_t i = base + it;
        if (i < n) out[i] = run;
        run += v[it];
    }
    // total goes to out[n] from the last block's last thread
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) out[n] = run;
}

__global__ void scan_single_k(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ out) {
    // one block, sequential over chunks of 1024 (used for short arrays)
    __shared__ int64_t carry;
    __shared__ int64_t wsum[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < n ? in[i] : 0;
        int lane = lane_id(), w = threadIdx.x >> 5;
        int64_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        int64_t woff = 0;
        for (int q = 0; q < w; ++q) woff += wsum[q];
        int64_t c = carry;
        if (i < n) out[i] = c + woff + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + woff + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry;
}

template <typename Tin>
static kc_status scan_impl(const Tin* in, int64_t* out, int64_t n, Arena& A, cudaStream_t s) {
    if (n <= 0) {
        KC_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return KC_OK;
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    int64_t* bsum;
    int64_t* boff;
    KC_TRY(A.get(&bsum, nb));
    KC_TRY(A.get(&boff, nb + 1));
    ::kc::note_launch(), scan_reduce_k<Tin><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bsum);
    if (nb <= 8192) ::kc::note_launch(), scan_single_k<<<1, 1024, 0, s>>>(bsum, nb, boff);
    else KC_TRY(scan_impl<int64_t>(bsum, boff, nb, A, s));
    ::kc::note_launch(), scan_tile_k<Tin><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, boff, out);
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

kc_status exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, Arena& A, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, A, s);
}
kc_status exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, Arena& A, cudaStream_t s) {
    return scan_impl<int32_t>(in, out, n, A, s);
}

// ------------------------------------------------------------ radix sort
// Tile of one block = 8 warps x 16 rounds x 32 lanes = 4096 elements, each
// warp owning 512 consecutive elements processed in order, so the scatter
// is stable.  Histograms are digit-major: hist[digit * ntiles + tile].
constexpr int RS_WARPS = 8;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_WARPS * RS_ROUNDS * 32;

template <typename K>
__global__ void rs_hist_k(const K* __restrict__ key, int64_t n, int shift, int64_t ntiles,
                          int64_t* __restrict__ hist) {
    __shared__ int cnt[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += blockDim.x) {
        int64_t e = base + i;
        if (e < n) atomicAdd(&cnt[(int)((key[e] >> shift) & 0xFF)], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[(int64_t)i * ntiles + blockIdx.x] = cnt[i];
}

// Scatter of one tile: each warp ranks its elements by digit once (match_any,
// in element order, so the sort is stable), keeping each element's key and
// its position among the warp's elements of the same digit in registers; the
// tile is then rearranged in shared memory in digit order, and every digit's
// run is written to its global offset with consecutive threads writing
// consecutive addresses.
template <typename K>
__global__ void __launch_bounds__(RS_WARPS * 32) rs_scatter_k(const K* __restrict__ kin, const int64_t* __restrict__ vin,
                                                               int64_t n, int shift, int64_t ntiles,
                                                               const int64_t* __restrict__ goff, K* __restrict__ kout,
                                                               int64_t* __restrict__ vout) {
    extern __shared__ __align__(16) unsigned char rs_smem[];
    int64_t* sval = (int64_t*)rs_smem;            // [RS_TILE]
    K* skey = (K*)(sval + RS_TILE);               // [RS_TILE]
    __shared__ int wcnt[RS_WARPS][256];           // per-warp digit counts, then the warps' starts in the tile
    __shared__ int dstart[257];                   // tile-local start of every digit
    __shared__ long long gbase[256];              // global start of every digit of this tile
    __shared__ int wsum[RS_WARPS];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    for (int i = lane; i < 256; i += 32) wcnt[w][i] = 0;
    __syncwarp();
    const int64_t tbase = (int64_t)blockIdx.x * RS_TILE;
    const int64_t wbase = tbase + (int64_t)w * RS_ROUNDS * 32;
    const unsigned lt = (1u << lane) - 1u;
    K kr[RS_ROUNDS];
    int rank[RS_ROUNDS];  // digit in the high bits, position among the warp's same-digit elements below
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int64_t e = wbase + r * 32 + lane;
        const bool ok = e < n;
        kr[r] = ok ? kin[e] : (K)0;
        const int dg = ok ? (int)((kr[r] >> shift) & 0xFF) : 256 + lane;
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const int before = ok ? wcnt[w][dg] : 0;
        __syncwarp();
        if (ok && lane == 31 - __clz(peers)) wcnt[w][dg] = before + __popc(peers);
        rank[r] = ok ? (dg << 16) | (before + __popc(peers & lt)) : -1;
        __syncwarp();
    }
    __syncthreads();
    // digit totals of the tile, their exclusive scan, and the per-warp offsets
    {
        const int dgt = threadIdx.x;  // blockDim == 256
        int tot = 0;
        for (int q = 0; q < RS_WARPS; ++q) tot += wcnt[q][dgt];
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        int off = 0;
        for (int q = 0; q < w; ++q) off += wsum[q];
        const int start = off + incl - tot;
        dstart[dgt] = start;
        if (dgt == 255) dstart[256] = start + tot;
        gbase[dgt] = goff[(int64_t)dgt * ntiles + blockIdx.x];
        int run = start;
        for (int q = 0; q < RS_WARPS; ++q) {
            const int c = wcnt[q][dgt];
            wcnt[q][dgt] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        if (rank[r] >= 0) {
            const int pos = wcnt[w][rank[r] >> 16] + (rank[r] & 0xFFFF);
            skey[pos] = kr[r];
            sval[pos] = vin[wbase + r * 32 + lane];
        }
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)RS_TILE, n - tbase);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const K kv = skey[i];
        const int dg = (int)((kv >> shift) & 0xFF);
        const long long pos = gbase[dg] + (i - dstart[dg]);
        kout[pos] = kv;
        vout[pos] = sval[i];
    }
}

template <typename K>
static size_t rs_smem_bytes() {
    return (size_t)RS_TILE * (sizeof(int64_t) + sizeof(K));
}

template <typename K>
static kc_status radix_impl(K* k_in, int64_t* v_in, K* k_out, int64_t* v_out, int64_t n, int bits, Arena& A,
                            cudaStream_t s) {
    if (n <= 0) return KC_OK;
    int passes = (bits + 7) / 8;
    if (passes < 1) passes = 1;
    KC_TRY(allow_dynamic_smem(rs_scatter_k<K>));
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    int64_t* hist;
    int64_t* goff;
    KC_TRY(A.get(&hist, 256 * ntiles));
    KC_TRY(A.get(&goff, 256 * ntiles + 1));
    K* ka = k_in;
    int64_t* va = v_in;
    K* kb = k_out;
    int64_t* vb = v_out;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        ::kc::note_launch(), rs_hist_k<K><<<(unsigned)ntiles, 256, 0, s>>>(ka, n, shift, ntiles, hist);
        KC_TRY(exclusive_scan_i64(hist, goff, 256 * ntiles, A, s));
        ::kc::note_launch(), rs_scatter_k<K><<<(unsigned)ntiles, RS_WARPS * 32, rs_smem_bytes<K>(), s>>>(
            ka, va, n, shift, ntiles, goff, kb, vb);
        KC_CUDA(cudaGetLastError());
        K* tk = ka; ka = kb; kb = tk;
        int64_t* tv = va; va = vb; vb = tv;
    }
    // after an odd number of passes the result is in the *_out buffers
    if (ka != k_out) {
        KC_CUDA(cudaMemcpyAsync(k_out, ka, sizeof(K) * n, cudaMemcpyDeviceToDevice, s));
        KC_CUDA(cudaMemcpyAsync(v_out, va, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    return KC_OK;
}

kc_status radix_sort_u64_i64(uint64_t* k_in, int64_t* v_in, uint64_t* k_out, int64_t* v_out, int64_t n, int bits,
                             Arena& A, cudaStream_t s) {
    return radix_impl<uint64_t>(k_in, v_in, k_out, v_out, n, bits, A, s);
}
kc_status radix_sort_u32_i64(uint32_t* k_in, int64_t* v_in, uint32_t* k_out, int64_t* v_out, int64_t n, int bits,
                             Arena& A, cudaStream_t s) {
    return radix_impl<uint32_t>(k_in, v_in, k_out, v_out, n, bits, A, s);
}

}  // namespace kc
