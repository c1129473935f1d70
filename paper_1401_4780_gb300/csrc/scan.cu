// scan.cu -- device-wide exclusive prefix sum of int64 (three passes: per-tile
// scans with their totals, one block over the tile totals, the add-back).
// Integer sums are exact, so the result does not depend on the tiling.
#include "common.cuh"
#include "scan.cuh"

namespace asyrk {

constexpr int SCAN_TILE = 2048;  // 256 threads x 8 items

__global__ void k_scan_tiles(const int64_t *__restrict__ in, int64_t *__restrict__ out,
                             int64_t *__restrict__ tile_sum, int64_t count)
{
    __shared__ int64_t part[SCAN_TILE / 8];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    const int t = threadIdx.x;  // 256 threads, 8 items each
    int64_t v[8], run = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int64_t q = base + t * 8 + k;
        v[k] = q < count ? in[q] : 0;
        run += v[k];
    }
    part[t] = run;
    __syncthreads();
    if (t == 0) {
        int64_t acc = 0;
        for (int w = 0; w < SCAN_TILE / 8; ++w) {
            const int64_t x = part[w];
            part[w] = acc;
            acc += x;
        }
        tile_sum[blockIdx.x] = acc;
    }
    __syncthreads();
    int64_t acc = part[t];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int64_t q = base + t * 8 + k;
        if (q < count) out[q] = acc;
        acc += v[k];
    }
}

// one block of 1024 threads scans the tile totals in chunks of 1024, carrying
// the running sum from chunk to chunk
__global__ void __launch_bounds__(1024) k_scan_sums(int64_t *__restrict__ tile_sum, int64_t tiles,
                                                    int64_t *__restrict__ total)
{
    __shared__ int64_t sh[1024];
    __shared__ int64_t carry;
    const int t = threadIdx.x;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < tiles; base += 1024) {
        const int64_t i = base + t;
        const int64_t v = i < tiles ? tile_sum[i] : 0;
        sh[t] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan (Hillis-Steele)
            const int64_t add = t >= o ? sh[t - o] : 0;
            __syncthreads();
            sh[t] += add;
            __syncthreads();
        }
        const int64_t c = carry;
        if (i < tiles) tile_sum[i] = c + sh[t] - v;
        __syncthreads();
        if (t == 1023) carry = c + sh[1023];
        __syncthreads();
    }
    if (t == 0) *total = carry;
}

__global__ void k_scan_add(int64_t *__restrict__ out, const int64_t *__restrict__ tile_sum,
                           int64_t count)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < count) out[q] += tile_sum[q / SCAN_TILE];
}

int64_t scan_tmp_count(int64_t count) { return (count + SCAN_TILE - 1) / SCAN_TILE + 1; }

int exclusive_scan(const int64_t *in, int64_t *out, int64_t count, int64_t *tmp, int64_t *total,
                   cudaStream_t s)
{
    const int64_t tiles = (count + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 0) {
        ASYRK_CK(cudaMemsetAsync(total, 0, sizeof(int64_t), s));
        return ASYRK_OK;
    }
    k_scan_tiles<<<(unsigned)tiles, 256, 0, s>>>(in, out, tmp, count);
    k_scan_sums<<<1, 1024, 0, s>>>(tmp, tiles, total);
    k_scan_add<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(out, tmp, count);
    ASYRK_CK(cudaGetLastError());
    return ASYRK_OK;
}

}  // namespace asyrk
