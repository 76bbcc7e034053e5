// primitives.cu -- device scan and radix sort used by the trie builder.
#include "eh_internal.cuh"

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

template <typename T>
__global__ void scan_tiles(const T *__restrict__ in, T *out, uint64_t n, T *block_sums) {
    __shared__ T warp_tot[SCAN_THREADS / 32];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T v[SCAN_ITEMS];
    T sum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        uint64_t idx = base + (uint64_t)tid * SCAN_ITEMS + i;
        v[i] = idx < n ? in[idx] : (T)0;
        sum += v[i];
    }
    T incl = warp_incl_scan(sum);
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = lane < SCAN_THREADS / 32 ? warp_tot[lane] : (T)0;
        T wi = warp_incl_scan(w);
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = wi - w;   // exclusive
    }
    __syncthreads();
    T run = incl - sum + warp_tot[warp];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        uint64_t idx = base + (uint64_t)tid * SCAN_ITEMS + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (tid == SCAN_THREADS - 1) block_sums[blockIdx.x] = run;
}

template <typename T>
__global__ void scan_add(T *out, uint64_t n, const T *__restrict__ offs) {
    uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) out[idx] += offs[idx / SCAN_TILE];
}

template <typename T>
eh_status scan_rec(const T *in, T *out, uint64_t n, cudaStream_t s) {
    if (n == 0) return EH_OK;
    uint64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    T *sums = nullptr;
    EH_TRY(dev_alloc(&sums, nb, s));
    scan_tiles<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, sums);
    eh_status st = EH_OK;
    if (nb > 1) {
        st = scan_rec<T>(sums, sums, nb, s);
        if (st == EH_OK) scan_add<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, sums);
    }
    dev_free(sums, s);
    return st;
}

template <typename T>
eh_status scan_total(const T *in, T *out, uint64_t n, cudaStream_t s, uint64_t *total_host) {
    if (n == 0) {
        if (total_host) *total_host = 0;
        return EH_OK;
    }
    T last_in = 0;
    if (total_host) EH_CUDA_TRY(cudaMemcpyAsync(&last_in, in + n - 1, sizeof(T), cudaMemcpyDeviceToHost, s));
    EH_TRY(scan_rec<T>(in, out, n, s));
    if (total_host) {
        EH_CUDA_TRY(cudaStreamSynchronize(s));   // last_in is ready, the scan is enqueued after it
        T last_out = 0;
        EH_CUDA_TRY(cudaMemcpyAsync(&last_out, out + n - 1, sizeof(T), cudaMemcpyDeviceToHost, s));
        EH_CUDA_TRY(cudaStreamSynchronize(s));
        *total_host = (uint64_t)last_out + (uint64_t)last_in;
    }
    EH_CUDA_TRY(cudaGetLastError());
    return EH_OK;
}

// ------------------------------------------------------------ radix sort

constexpr int RS_THREADS = 512;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 5;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_BINS = 256;

__global__ void __launch_bounds__(RS_THREADS) rs_upsweep(const uint64_t *__restrict__ keys, uint64_t n, uint64_t chunk,
                                                           int shift, uint32_t dmask, uint32_t *hist) {
    __shared__ uint32_t h[RS_BINS];
    const int tid = threadIdx.x;
    for (int b = tid; b < RS_BINS; b += RS_THREADS) h[b] = 0;
    __syncthreads();
    uint64_t begin = (uint64_t)blockIdx.x * chunk;
    uint64_t end = begin + chunk < n ? begin + chunk : n;
    for (uint64_t i = begin + tid; i < end; i += RS_THREADS) atomicAdd(&h[(keys[i] >> shift) & dmask], 1u);
    __syncthreads();
    for (int b = tid; b < RS_BINS; b += RS_THREADS) hist[(uint64_t)b * gridDim.x + blockIdx.x] = h[b];
}

// Stable scatter of one digit of up to 8 bits (dmask).  Per tile: every warp
// ranks its keys among the keys of the same digit (match_any, in input order), the tile's
// keys are placed in digit order in shared memory, and each digit's run is
// then written to its global range with consecutive threads on consecutive
// addresses (coalesced), instead of one scattered store per key.
__global__ void __launch_bounds__(RS_THREADS) rs_downsweep(const uint64_t *__restrict__ in, uint64_t *__restrict__ out,
                                                             uint64_t n, uint64_t chunk, int shift, uint32_t dmask,
                                                             const uint32_t *__restrict__ offs) {
    __shared__ uint32_t wcnt[RS_WARPS][RS_BINS];   // per-warp digit counts, then the warps' offsets in the digit's run
    __shared__ uint32_t run[RS_BINS];              // global position of the digit's next key
    __shared__ uint32_t loc[RS_BINS];              // tile-local start of the digit's run
    __shared__ uint64_t skey[RS_TILE];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int b = tid; b < RS_BINS; b += RS_THREADS) run[b] = offs[(uint64_t)b * gridDim.x + blockIdx.x];
    uint64_t begin = (uint64_t)blockIdx.x * chunk;
    uint64_t end = begin + chunk < n ? begin + chunk : n;
    for (uint64_t tile = begin; tile < end; tile += RS_TILE) {
        for (int i = 0; i < RS_WARPS; ++i)
            for (int b = tid; b < RS_BINS; b += RS_THREADS) wcnt[i][b] = 0;
        __syncthreads();
        const uint64_t sub = tile + (uint64_t)warp * 32 * RS_ITEMS;
        uint64_t k[RS_ITEMS];
        uint32_t dig[RS_ITEMS], wr[RS_ITEMS];
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r) {
            const uint64_t idx = sub + (uint64_t)r * 32 + lane;
            const bool valid = idx < end;
            k[r] = valid ? in[idx] : 0ull;
            dig[r] = valid ? (uint32_t)(k[r] >> shift) & dmask : 256u;   // 256: no key
            const uint32_t peers = __match_any_sync(0xffffffffu, dig[r]);
            const uint32_t before = valid ? wcnt[warp][dig[r]] : 0u;     // this warp's earlier keys of the digit
            __syncwarp();
            wr[r] = before + __popc(peers & lt_mask);
            if (valid && (peers & lt_mask) == 0) wcnt[warp][dig[r]] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        for (int b = tid; b < RS_BINS; b += RS_THREADS) {
            uint32_t c = 0;
            for (int w = 0; w < RS_WARPS; ++w) {
                const uint32_t x = wcnt[w][b];
                wcnt[w][b] = c;
                c += x;
            }
            loc[b] = c;   // the digit's total in the tile, scanned next
        }
        __syncthreads();
        if (warp == 0) {   // exclusive scan of the 256 totals, 8 per lane
            uint32_t v[8], sum = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) { v[i] = loc[lane * 8 + i]; sum += v[i]; }
            uint32_t incl = sum;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            uint32_t ex = incl - sum;
#pragma unroll
            for (int i = 0; i < 8; ++i) { loc[lane * 8 + i] = ex; ex += v[i]; }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r)
            if (dig[r] < 256u) skey[loc[dig[r]] + wcnt[warp][dig[r]] + wr[r]] = k[r];
        __syncthreads();
        const uint32_t cnt = (uint32_t)(end - tile < (uint64_t)RS_TILE ? end - tile : (uint64_t)RS_TILE);
        for (uint32_t i = tid; i < cnt; i += RS_THREADS) {
            const uint64_t key = skey[i];
            const uint32_t d = (uint32_t)(key >> shift) & dmask;
            out[run[d] + (i - loc[d])] = key;
        }
        __syncthreads();
        for (int b = tid; b < RS_BINS; b += RS_THREADS) run[b] += (b < RS_BINS - 1 ? loc[b + 1] : cnt) - loc[b];
        __syncthreads();
    }
}

}  // namespace

eh_status dev_exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint64_t n, cudaStream_t s,
                                 uint64_t *total_host) {
    return scan_total<uint32_t>(in, out, n, s, total_host);
}

eh_status dev_exclusive_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, cudaStream_t s,
                                 uint64_t *total_host) {
    return scan_total<uint64_t>(in, out, n, s, total_host);
}

eh_status dev_radix_sort_u64(uint64_t **keys, uint64_t **tmp, uint64_t n, int key_bits, cudaStream_t s) {
    if (n <= 1 || key_bits <= 0) return EH_OK;
    if (n >= (1ull << 32)) {
        eh_set_error("radix sort: %llu keys exceed the 32-bit rank range", (unsigned long long)n);
        return EH_EINVAL;
    }
    uint64_t tiles = (n + RS_TILE - 1) / RS_TILE;
    uint64_t G = (uint64_t)eh_num_sms() * 4;
    if (G > tiles) G = tiles;
    if (G < 1) G = 1;
    uint64_t chunk = (tiles + G - 1) / G * RS_TILE;
    G = (n + chunk - 1) / chunk;
    uint32_t *hist = nullptr;
    EH_TRY(dev_alloc(&hist, RS_BINS * G, s));
    eh_status st = EH_OK;
    for (int shift = 0; shift < key_bits; shift += 8) {
        // the last digit keeps only the bits below key_bits: bits above them
        // need not be zero (a sort on the low field of a packed key)
        const uint32_t dmask = key_bits - shift >= 8 ? 255u : (1u << (key_bits - shift)) - 1u;
        rs_upsweep<<<(unsigned)G, RS_THREADS, 0, s>>>(*keys, n, chunk, shift, dmask, hist);
        st = dev_exclusive_scan_u32(hist, hist, RS_BINS * G, s, nullptr);
        if (st != EH_OK) break;
        rs_downsweep<<<(unsigned)G, RS_THREADS, 0, s>>>(*keys, *tmp, n, chunk, shift, dmask, hist);
        uint64_t *t = *keys;
        *keys = *tmp;
        *tmp = t;
    }
    dev_free(hist, s);
    EH_CUDA_TRY(cudaGetLastError());
    return st;
}
