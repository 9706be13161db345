// Layout preparation (S0): re-lays the caller's canonical FP64 blocks into the
// K-major operand layouts of the W-contraction kernels, zero-padding K, and
// for the mixed precisions splits each value x into hi = round(x) and
// lo = round(x - hi) in TF32 or BF16 (the split-precision scheme that replaces
// the paper's dgemm -> sgemm swap of Sec. 3).
#include <cuda_bf16.h>

#include "tcorr_internal.cuh"

namespace tcorr {
namespace {

constexpr int TT = 32;  // transpose tile edge

__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r & 0xFFFFE000u);  // TF32 keeps 10 mantissa bits
}

template <int KIND>
__device__ __forceinline__ void store_split(void *hi, void *lo, int64_t idx, double x) {
    if constexpr (KIND == 0) {
        static_cast<double *>(hi)[idx] = x;
    } else if constexpr (KIND == 1) {
        const float h = tf32_rn(static_cast<float>(x));
        const float l = tf32_rn(static_cast<float>(x - static_cast<double>(h)));
        static_cast<float *>(hi)[idx] = h;
        static_cast<float *>(lo)[idx] = l;
    } else {
        const __nv_bfloat16 h = __double2bfloat16(x);
        const __nv_bfloat16 l = __double2bfloat16(x - static_cast<double>(__bfloat162float(h)));
        static_cast<__nv_bfloat16 *>(hi)[idx] = h;
        static_cast<__nv_bfloat16 *>(lo)[idx] = l;
    }
}

// One CTA (32 x 8 threads) moves a TT x TT tile: rows r (output-contiguous),
// columns c (input-contiguous when sc = 1).  Tiles are enumerated flat over
// (b, c-tile, r-tile) in blockIdx.x (64-bit safe through a grid-stride loop).
template <int KIND>
__global__ void __launch_bounds__(256) transpose_pad_kernel(
    const double *__restrict__ in, void *out_hi, void *out_lo, int64_t B, int R, int Rp,
    int64_t C, int64_t sb, int64_t sr, int64_t sc, int64_t ob, int64_t oc, double scale) {
    __shared__ double tile[TT][TT + 1];
    const int64_t nct = (C + TT - 1) / TT;
    const int64_t nrt = (Rp + TT - 1) / TT;
    const int64_t ntiles = B * nct * nrt;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t rt = t % nrt;
        const int64_t ct = (t / nrt) % nct;
        const int64_t b = t / (nrt * nct);
        const int64_t r0 = rt * TT, c0 = ct * TT;
        // load: column c0+tx, rows r0+ty+8m
        for (int m = 0; m < TT; m += 8) {
            const int64_t r = r0 + ty + m, c = c0 + tx;
            double x = 0.0;
            if (r < R && c < C) x = scale * in[b * sb + r * sr + c * sc];
            tile[ty + m][tx] = x;
        }
        __syncthreads();
        // store: row c0+ty+8m of the output, element r0+tx
        for (int m = 0; m < TT; m += 8) {
            const int64_t c = c0 + ty + m, r = r0 + tx;
            if (c < C && r < Rp) store_split<KIND>(out_hi, out_lo, b * ob + c * oc + r, tile[tx][ty + m]);
        }
        __syncthreads();
    }
}

// FP32 epilogue inputs of the split-precision paths, the virtual extents
// padded with zeros to vp (a multiple of the epilogue's cube edge 8): (p x | q z)
// as [p][q][X][Z][8][8], so that each of an orbit's 8x8 sub-blocks is one
// contiguous, aligned 256-byte bulk copy, and t1 as rows [p][x].
__global__ void ovov_blocks_kernel(const double *__restrict__ in, float *__restrict__ out, int o, int v,
                                   int vp) {
    const int64_t n = (int64_t)o * o * vp * vp;
    const int nb = vp / 8;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int lz = (int)(i & 7), lx = (int)((i >> 3) & 7);
        int64_t r = i >> 6;
        const int zb = (int)(r % nb);
        r /= nb;
        const int xb = (int)(r % nb);
        r /= nb;
        const int q = (int)(r % o), pp = (int)(r / o);
        const int x = xb * 8 + lx, z = zb * 8 + lz;
        out[i] = (x < v && z < v) ? static_cast<float>(in[(((int64_t)pp * v + x) * o + q) * v + z]) : 0.f;
    }
}

// eps_v as float-float pairs: hi = eps rounded to FP32, lo = the rest rounded
// to FP32 (about 48 significant bits together); zero for x >= v
__global__ void eps_ff_kernel(const double *__restrict__ e, float2 *__restrict__ out, int v, int vp) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= vp) return;
    const double d = x < v ? e[x] : 0.0;
    const float hi = static_cast<float>(d);
    out[x] = make_float2(hi, static_cast<float>(d - static_cast<double>(hi)));
}

// FP64 values to float-float pairs in place (the same 8 bytes per value)
__global__ void to_ff_kernel(double *__restrict__ x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = x[i];
        const float hi = static_cast<float>(d);
        reinterpret_cast<float2 *>(x)[i] = make_float2(hi, static_cast<float>(d - static_cast<double>(hi)));
    }
}

__global__ void pad_rows_kernel(const double *__restrict__ in, float *__restrict__ out, int rows, int v,
                                int vp) {
    const int64_t n = (int64_t)rows * vp;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % vp);
        out[i] = x < v ? static_cast<float>(in[(i / vp) * v + x]) : 0.f;
    }
}

}  // namespace

cudaError_t launch_transpose_pad(int kind, const double *in, void *out_hi, void *out_lo,
                                 int64_t B, int R, int Rp, int64_t C, int64_t sb, int64_t sr,
                                 int64_t sc, int64_t ob, int64_t oc, double scale,
                                 cudaStream_t st) {
    const int64_t ntiles = B * ((C + TT - 1) / TT) * ((Rp + TT - 1) / TT);
    if (ntiles == 0) return cudaSuccess;
    const unsigned grid = (unsigned)(ntiles < (int64_t)1 << 22 ? ntiles : (int64_t)1 << 22);
    dim3 blk(TT, 8);
    if (kind == 0)
        transpose_pad_kernel<0><<<grid, blk, 0, st>>>(in, out_hi, out_lo, B, R, Rp, C, sb, sr, sc,
                                                      ob, oc, scale);
    else if (kind == 1)
        transpose_pad_kernel<1><<<grid, blk, 0, st>>>(in, out_hi, out_lo, B, R, Rp, C, sb, sr, sc,
                                                      ob, oc, scale);
    else
        transpose_pad_kernel<2><<<grid, blk, 0, st>>>(in, out_hi, out_lo, B, R, Rp, C, sb, sr, sc,
                                                      ob, oc, scale);
    return cudaGetLastError();
}

cudaError_t launch_epilogue_ff_inputs(double *t1, double *ovov, const double *eps_v, float2 *evf, int o, int v,
                                      cudaStream_t st) {
    const int64_t n = (int64_t)o * v * o * v, blocks = (n + 255) / 256;
    to_ff_kernel<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, st>>>(ovov, n);
    to_ff_kernel<<<(unsigned)(((int64_t)o * v + 255) / 256), 256, 0, st>>>(t1, (int64_t)o * v);
    eps_ff_kernel<<<(v + 255) / 256, 256, 0, st>>>(eps_v, evf, v, v);
    return cudaGetLastError();
}

cudaError_t launch_epilogue_f32_inputs(const double *t1, const double *ovov, const double *eps_v, float *t1f,
                                       float *ovf, float2 *evf, int o, int v, int vp, cudaStream_t st) {
    if (vp % 8 != 0 || vp < v) return cudaErrorInvalidValue;
    const int64_t n = (int64_t)o * o * vp * vp, blocks = (n + 255) / 256;
    ovov_blocks_kernel<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, st>>>(ovov, ovf, o, v, vp);
    pad_rows_kernel<<<(unsigned)((o * (int64_t)vp + 255) / 256), 256, 0, st>>>(t1, t1f, o, v, vp);
    eps_ff_kernel<<<(vp + 255) / 256, 256, 0, st>>>(eps_v, evf, v, vp);
    return cudaGetLastError();
}


namespace {
// Thread per leading index x: the sorted triples x <= y <= z of n values
// start at offset sum_{x' < x} (n - x')(n - x' + 1) / 2.
__global__ void sorted_triples_kernel(int n, int *out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    int64_t off = 0;
    for (int xp = 0; xp < x; xp++) off += (int64_t)(n - xp) * (n - xp + 1) / 2;
    int *w = out + 3 * off;
    for (int y = x; y < n; y++)
        for (int z = y; z < n; z++) {
            w[0] = x;
            w[1] = y;
            w[2] = z;
            w += 3;
        }
}
}  // namespace

cudaError_t launch_build_tables(int o, int nb, int *tasks, int *orbits, cudaStream_t st) {
    sorted_triples_kernel<<<(o + 63) / 64, 64, 0, st>>>(o, tasks);
    sorted_triples_kernel<<<(nb + 63) / 64, 64, 0, st>>>(nb, orbits);
    return cudaGetLastError();
}

}  // namespace tcorr
