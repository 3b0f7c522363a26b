// pc_util.cu -- device buffers, errors, device-wide scan and i128 reduction.
#include <cstdarg>
#include <cstring>

#include "pc_internal.h"

void pc_set_error(pc_ctx* ctx, const char* fmt, ...)
{
    if (!ctx) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->errmsg, sizeof(ctx->errmsg), fmt, ap);
    va_end(ap);
}

int buf_reserve(pc_ctx* ctx, DevBuf& b, size_t bytes)
{
    if (bytes <= b.bytes && b.p) return PC_OK;
    if (ctx->mq_mode == MQ_CAPTURE) {   // captured nodes may already point at b.p
        pc_set_error(ctx, "internal: scratch of %zu bytes grown during graph capture", bytes);
        return PC_EINVAL;
    }
    if (b.p) {
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    size_t want = bytes < 256 ? 256 : bytes;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        pc_set_error(ctx, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
        return PC_ENOMEM;
    }
    b.bytes = want;
    return PC_OK;
}

void buf_free(DevBuf& b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

int copy_to_host(pc_ctx* ctx, void* dst, const void* src, size_t bytes)
{
    PC_CUDA(ctx, cudaMemcpyAsync(ctx->host_stage, src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    PC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    memcpy(dst, ctx->host_stage, bytes);
    return PC_OK;
}

// ------------------------------------------------------------------- scan
// Three-phase exclusive scan: tile sums, one-CTA scan of the tile sums, then
// per-tile scans with the tile offset.  TILE elements per CTA of 256 threads.
static constexpr int SCAN_THREADS = 256;
static constexpr int SCAN_PER = 8;
static constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER;

template <class TO>
__global__ void scan_tile_sums(const u32* in, u64 n, TO* sums)
{
    __shared__ TO sh[SCAN_THREADS / 32];
    u64 base = (u64)blockIdx.x * SCAN_TILE;
    TO s = 0;
    for (int k = 0; k < SCAN_PER; k++) {
        u64 i = base + (u64)k * SCAN_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        TO t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; w++) t += sh[w];
        sums[blockIdx.x] = t;
    }
}

// exclusive scan of sums[0..m) in place, one CTA; sums[m] = total
template <class TO>
__global__ void scan_sums_one_cta(TO* sums, u64 m)
{
    __shared__ TO wsum[SCAN_THREADS / 32];
    __shared__ TO carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (u64 base = 0; base < m; base += SCAN_THREADS) {
        u64 i = base + threadIdx.x;
        TO v = i < m ? sums[i] : 0;
        TO incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            TO t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            TO w = lane < SCAN_THREADS / 32 ? wsum[lane] : 0;
            TO wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                TO t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            if (lane < SCAN_THREADS / 32) wsum[lane] = wi - w;
        }
        __syncthreads();
        TO c0 = carry;
        if (i < m) sums[i] = c0 + wsum[wid] + incl - v;
        __syncthreads();
        if (threadIdx.x == SCAN_THREADS - 1) carry = c0 + wsum[wid] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[m] = carry;
}

template <class TO>
__global__ void scan_tiles(const u32* in, TO* out, u64 n, const TO* sums)
{
    __shared__ TO wsum[SCAN_THREADS / 32];
    __shared__ TO carry;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = sums[blockIdx.x];
    __syncthreads();
    u64 base = (u64)blockIdx.x * SCAN_TILE;
    for (int k = 0; k < SCAN_PER; k++) {
        u64 i = base + (u64)k * SCAN_THREADS + threadIdx.x;
        TO v = i < n ? (TO)in[i] : 0;
        TO incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            TO t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            TO w = lane < SCAN_THREADS / 32 ? wsum[lane] : 0;
            TO wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                TO t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            if (lane < SCAN_THREADS / 32) wsum[lane] = wi - w;
        }
        __syncthreads();
        TO c0 = carry;
        if (i < n) out[i] = c0 + wsum[wid] + incl - v;
        __syncthreads();
        if (threadIdx.x == SCAN_THREADS - 1) carry = c0 + wsum[wid] + incl;
        __syncthreads();
    }
}

template <class TO>
__global__ void scan_write_total(TO* out, u64 n, const TO* sums, u64 m)
{
    out[n] = sums[m];
}

template <class TO>
static int scan_impl(pc_ctx* ctx, const u32* in, TO* out, u64 n)
{
    u64 tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 0) tiles = 1;
    PC_TRY(buf_reserve(ctx, ctx->scan_tmp, (tiles + 1) * sizeof(TO)));
    TO* sums = ctx->scan_tmp.as<TO>();
    if (!mq_device_work(ctx)) return PC_OK;
    scan_tile_sums<TO><<<(unsigned)tiles, SCAN_THREADS, 0, ctx->stream>>>(in, n, sums);
    PC_LAUNCHED(ctx);
    scan_sums_one_cta<TO><<<1, SCAN_THREADS, 0, ctx->stream>>>(sums, tiles);
    PC_LAUNCHED(ctx);
    scan_tiles<TO><<<(unsigned)tiles, SCAN_THREADS, 0, ctx->stream>>>(in, out, n, sums);
    PC_LAUNCHED(ctx);
    scan_write_total<TO><<<1, 1, 0, ctx->stream>>>(out, n, sums, tiles);
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches += 4;
    return PC_OK;
}

int scan_exclusive_u32_to_u32(pc_ctx* ctx, const u32* in, u32* out, u64 n)
{
    return scan_impl<u32>(ctx, in, out, n);
}

int scan_exclusive_u32_to_u64(pc_ctx* ctx, const u32* in, u64* out, u64 n)
{
    return scan_impl<u64>(ctx, in, out, n);
}

// --------------------------------------------------------- i128 reduction
__global__ void reduce_i128_kernel(const I128Pair* in, u64 n, I128Pair* out)
{
    __shared__ i128 scratch[32];
    i128 s = 0;
    for (u64 i = threadIdx.x; i < n; i += blockDim.x) s += load_i128(in + i);
    s = block_sum_i128(s, scratch);
    if (threadIdx.x == 0) store_i128(out, load_i128(out) + s);
}

// *out += sum(in[0..n))
int reduce_i128(pc_ctx* ctx, const I128Pair* in, u64 n, I128Pair* out)
{
    reduce_i128_kernel<<<1, 1024, 0, ctx->stream>>>(in, n, out);
    PC_LAUNCHED(ctx);
    ctx->stats.kernel_launches += 1;
    return PC_OK;
}
