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

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 12;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__global__ void rs_upsweep(const uint64_t *__restrict__ keys, uint64_t n, uint64_t chunk, int shift,
                           uint32_t *hist) {
    __shared__ uint32_t h[256];
    const int tid = threadIdx.x;
    h[tid] = 0;
    __syncthreads();
    uint64_t begin = (uint64_t)blockIdx.x * chunk;
    uint64_t end = begin + chunk < n ? begin + chunk : n;
    for (uint64_t i = begin + tid; i < end; i += RS_THREADS) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(uint64_t)tid * gridDim.x + blockIdx.x] = h[tid];
}

__global__ void rs_downsweep(const uint64_t *__restrict__ in, uint64_t *__restrict__ out, uint64_t n,
                             uint64_t chunk, int shift, const uint32_t *__restrict__ offs) {
    __shared__ uint32_t whist[RS_WARPS][256];
    __shared__ uint32_t run[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    run[tid] = offs[(uint64_t)tid * gridDim.x + blockIdx.x];
    uint64_t begin = (uint64_t)blockIdx.x * chunk;
    uint64_t end = begin + chunk < n ? begin + chunk : n;
    for (uint64_t tile = begin; tile < end; tile += RS_TILE) {
#pragma unroll
        for (int i = 0; i < RS_WARPS; ++i) whist[i][tid] = 0;
        __syncthreads();
        const uint64_t sub = tile + (uint64_t)warp * 32 * RS_ITEMS;
        uint64_t k[RS_ITEMS];
        uint32_t dig[RS_ITEMS];
        uint32_t pm[RS_ITEMS];   // lanes of the warp holding the same digit (kept for the scatter)
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r) {
            uint64_t idx = sub + (uint64_t)r * 32 + lane;
            bool valid = idx < end;
            k[r] = valid ? in[idx] : 0ull;
            dig[r] = valid ? (uint32_t)(k[r] >> shift) & 255u : 256u;   // 256: no key
            pm[r] = __match_any_sync(0xffffffffu, dig[r]);
            if (valid && (pm[r] & lt_mask) == 0) whist[warp][dig[r]] += __popc(pm[r]);
            __syncwarp();
        }
        __syncthreads();
        {
            uint32_t r0 = run[tid];
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) {
                uint32_t c = whist[w][tid];
                whist[w][tid] = r0;
                r0 += c;
            }
            run[tid] = r0;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < RS_ITEMS; ++r) {
            const bool valid = dig[r] < 256u;
            const uint32_t peers = pm[r];
            uint32_t base = valid ? whist[warp][dig[r]] : 0u;
            __syncwarp();
            if (valid) {
                out[base + __popc(peers & lt_mask)] = k[r];
                if ((peers & lt_mask) == 0) whist[warp][dig[r]] = base + __popc(peers);
            }
            __syncwarp();
        }
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
    uint64_t G = (uint64_t)eh_num_sms() * 8;
    if (G > tiles) G = tiles;
    if (G < 1) G = 1;
    uint64_t chunk = (tiles + G - 1) / G * RS_TILE;
    G = (n + chunk - 1) / chunk;
    uint32_t *hist = nullptr;
    EH_TRY(dev_alloc(&hist, 256 * G, s));
    eh_status st = EH_OK;
    for (int shift = 0; shift < key_bits; shift += 8) {
        rs_upsweep<<<(unsigned)G, RS_THREADS, 0, s>>>(*keys, n, chunk, shift, hist);
        st = dev_exclusive_scan_u32(hist, hist, 256 * G, s, nullptr);
        if (st != EH_OK) break;
        rs_downsweep<<<(unsigned)G, RS_THREADS, 0, s>>>(*keys, *tmp, n, chunk, shift, hist);
        uint64_t *t = *keys;
        *keys = *tmp;
        *tmp = t;
    }
    dev_free(hist, s);
    EH_CUDA_TRY(cudaGetLastError());
    return st;
}
