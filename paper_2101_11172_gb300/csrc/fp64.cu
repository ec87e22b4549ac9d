// FP64 path of gridding and degridding (plans made with WS_FLAG_FP64).
//
// The single-precision path is limited by FP32 rounding near 3e-7 relative,
// while the method's own bound E falls far lower for wider kernels (E of
// Eq. norm_bound is 6e-13 at W = 12 and reaches double-precision level at
// W = 14, x0 = 1/4; Section 6.3).  This path keeps everything in FP64 --
// coordinates, weights (the Chebyshev series of the plan's fit, evaluated
// by Clenshaw's recurrence), the w-stack, the plane transforms, the screens
// and the sums -- so that its error against the exact DFT follows sqrt(3) E
// down to W = 14.  It exists to measure the method's error, not for
// throughput: each w-plane is taken on its own with plain kernels (FP64
// atomics for the spread, a radix-2 shared-memory FFT per line), Algorithm 5
// and Algorithm 6 step by step.
//
// Layout: one N' x N' plane of complex128, row S (v) by column R (u), both
// modulo N' as in the FP32 path; images N x N complex128; visibilities
// complex128.
#include <math.h>

#include <algorithm>

#include "ws_internal.hpp"

namespace ws {
namespace {

struct VisRec64 {
    int r0, s0, t0, folded;     // t0 < 0: dropped
    double nux, nuy, nuz;
    double pre_re, pre_im;      // exp(+2 pi i w (n0 - 1))
};

__device__ __forceinline__ int wrap_index64(double x, int n) {
    long long i = (long long)x;
    if (i < -n || i >= 2LL * n) i %= n;
    if (i < 0) i += n;
    if (i >= n) i -= n;
    return (int)i;
}

// c_i(nu) = sum_k cheb[i][k] T_k(2 nu) by Clenshaw's recurrence.
__device__ __forceinline__ double tap_weight(const double *__restrict__ cheb, int deg, int i, double nu) {
    const double *c = cheb + (size_t)i * (deg + 1);
    const double y = 2.0 * nu;
    double b1 = 0.0, b2 = 0.0;
    for (int k = deg; k >= 1; --k) {
        const double b0 = 2.0 * y * b1 - b2 + c[k];
        b2 = b1;
        b1 = b0;
    }
    return y * b1 - b2 + c[0];
}

__global__ void prep64_kernel(Launch L, const double *__restrict__ uvw, int64_t M, VisRec64 *__restrict__ rec,
                              unsigned long long *__restrict__ drop) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    double u = uvw[3 * k], v = uvw[3 * k + 1], w = uvw[3 * k + 2];
    const bool folded = L.fold && w < 0.0;     // Section 5.4: conjugate visibility at -(u, v, w)
    if (folded) {
        u = -u;
        v = -v;
        w = -w;
    }
    const int W = L.W;
    VisRec64 r{0, 0, -1, folded ? 1 : 0, 0.0, 0.0, 0.0, 1.0, 0.0};
    const double up = u * L.uv_scale, vp = v * L.uv_scale, wp = w * L.nscale;
    if (!(fabs(up) < 1e15) || !(fabs(vp) < 1e15)) {
        atomicAdd(&drop[0], 1ull);
        rec[k] = r;
        return;
    }
    const double ft = floor(wp + 0.5 * W);
    const double t0 = ft - (W - 1) - L.t_lo;
    if (!(t0 >= 0.0 && t0 + W <= (double)L.Nw)) {
        atomicAdd(&drop[1], 1ull);
        rec[k] = r;
        return;
    }
    const double fu = floor(up + 0.5 * W), fv = floor(vp + 0.5 * W);
    r.r0 = wrap_index64(fu - (W - 1), L.Np);
    r.s0 = wrap_index64(fv - (W - 1), L.Np);
    r.t0 = (int)t0;
    r.nux = up + 0.5 * (W - 1) - fu;
    r.nuy = vp + 0.5 * (W - 1) - fv;
    r.nuz = wp + 0.5 * (W - 1) - ft;
    double turns = w * L.n0m1;
    turns -= rint(turns);
    sincospi(2.0 * turns, &r.pre_im, &r.pre_re);
    rec[k] = r;
}

// Algorithm 5 steps 2-3a for plane p: every visibility whose footprint
// includes p adds V exp(2 pi i w (n0-1)) C_x C_y C_z(p - t0) to its W x W cells.
__global__ void spread64_kernel(Launch L, const double *__restrict__ cheb, int deg, const VisRec64 *__restrict__ rec,
                                const double2 *__restrict__ vis, int64_t M, int p, double2 *__restrict__ plane) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    const VisRec64 r = rec[k];
    const int c = p - r.t0;
    if (r.t0 < 0 || c < 0 || c >= L.W) return;
    double2 V = vis[k];
    if (r.folded) V.y = -V.y;
    const double vr = V.x * r.pre_re - V.y * r.pre_im, vi = V.x * r.pre_im + V.y * r.pre_re;
    const double wz = tap_weight(cheb + (size_t)L.W * (deg + 1), deg, c, r.nuz);
    double wx[kMaxW64];
    for (int a = 0; a < L.W; ++a) wx[a] = tap_weight(cheb, deg, a, r.nux);
    const int Np = L.Np;
    for (int b = 0; b < L.W; ++b) {
        const double wyz = tap_weight(cheb, deg, b, r.nuy) * wz;
        double *row = reinterpret_cast<double *>(plane + (size_t)((r.s0 + b) % Np) * Np);
        for (int a = 0; a < L.W; ++a) {
            const int R = (r.r0 + a) % Np;
            atomicAdd(row + 2 * R, vr * wyz * wx[a]);
            atomicAdd(row + 2 * R + 1, vi * wyz * wx[a]);
        }
    }
}

// Radix-2 decimation-in-time FFT of one line of n = 2^logn points in shared
// memory; line l of the plane starts at l * line_stride and its points are
// elem_stride apart.  tw[m] = exp(-2 pi i m / n) (FP64 table), sign +1 for
// the inverse transform.  One CTA per line.
__global__ void fft64_lines_kernel(double2 *__restrict__ plane, int n, int logn, size_t line_stride,
                                   size_t elem_stride, const double2 *__restrict__ tw, int inverse) {
    extern __shared__ double2 buf64[];
    double2 *line = plane + (size_t)blockIdx.x * line_stride;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int rev = (int)(__brev((unsigned)i) >> (32 - logn));
        buf64[rev] = line[(size_t)i * elem_stride];
    }
    __syncthreads();
    for (int half = 1, s = 0; half < n; half <<= 1, ++s) {
        const int shift = logn - 1 - s;               // twiddle step n / (2 half)
        for (int q = threadIdx.x; q < n / 2; q += blockDim.x) {
            const int j = q & (half - 1), base = (q - j) * 2 + j;
            double2 w = tw[j << shift];
            if (inverse) w.y = -w.y;
            const double2 a = buf64[base], b = buf64[base + half];
            const double2 bw = make_double2(b.x * w.x - b.y * w.y, b.x * w.y + b.y * w.x);
            buf64[base] = make_double2(a.x + bw.x, a.y + bw.y);
            buf64[base + half] = make_double2(a.x - bw.x, a.y - bw.y);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) line[(size_t)i * elem_stride] = buf64[i];
}

__device__ __forceinline__ int crop64(int c, int half, int Np) { return c < half ? c - half + Np : c - half; }

// Algorithm 5 steps 3c-4: crop, exp(+2 pi i t z), sum over planes.
__global__ void crop_acc64_kernel(Launch L, const double2 *__restrict__ plane, const double *__restrict__ z,
                                  double t, double2 *__restrict__ acc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int N = L.N;
    if (i >= (int64_t)N * N) return;
    const int row = (int)(i / N), col = (int)(i % N);
    const double2 P = plane[(size_t)crop64(row, N / 2, L.Np) * L.Np + crop64(col, N / 2, L.Np)];
    double tz = t * z[i];
    tz -= rint(tz);
    double s, c;
    sincospi(2.0 * tz, &s, &c);
    acc[i] = make_double2(acc[i].x + P.x * c - P.y * s, acc[i].y + P.x * s + P.y * c);
}

// Algorithm 5 step 5: dirty = h_x h_y h_z D (real part only for a folded real-sky plan).
__global__ void finish_grid64_kernel(int64_t n, const double *__restrict__ corr, const double2 *__restrict__ acc,
                                     int fold, double2 *__restrict__ dirty) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dirty[i] = make_double2(corr[i] * acc[i].x, fold ? 0.0 : corr[i] * acc[i].y);
}

// Algorithm 6 steps 3a-3b: the plane's padded, screened, corrected image.
__global__ void pad_screen64_kernel(Launch L, const double *__restrict__ corr, const double2 *__restrict__ image,
                                    const double *__restrict__ z, double t, double2 *__restrict__ plane) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int N = L.N;
    if (i >= (int64_t)N * N) return;
    const int row = (int)(i / N), col = (int)(i % N);
    const double2 f = image[i];
    const double fr = corr[i] * f.x, fi = L.fold ? 0.0 : corr[i] * f.y;
    double tz = t * z[i];
    tz -= rint(tz);
    double s, c;
    sincospi(2.0 * tz, &s, &c);
    plane[(size_t)crop64(row, N / 2, L.Np) * L.Np + crop64(col, N / 2, L.Np)] =
        make_double2(fr * c + fi * s, fi * c - fr * s);
}

// Algorithm 6 step 4 for plane p: the visibilities whose footprint includes p
// add C_z(p - t0) sum_{a,b} F C_x C_y.
__global__ void gather64_kernel(Launch L, const double *__restrict__ cheb, int deg, const VisRec64 *__restrict__ rec,
                                int64_t M, int p, const double2 *__restrict__ plane, double2 *__restrict__ acc) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    const VisRec64 r = rec[k];
    const int c = p - r.t0;
    if (r.t0 < 0 || c < 0 || c >= L.W) return;
    const double wz = tap_weight(cheb + (size_t)L.W * (deg + 1), deg, c, r.nuz);
    double wx[kMaxW64];
    for (int a = 0; a < L.W; ++a) wx[a] = tap_weight(cheb, deg, a, r.nux);
    const int Np = L.Np;
    double sr = 0.0, si = 0.0;
    for (int b = 0; b < L.W; ++b) {
        const double wy = tap_weight(cheb, deg, b, r.nuy);
        const double2 *row = plane + (size_t)((r.s0 + b) % Np) * Np;
        double rr = 0.0, ri = 0.0;
        for (int a = 0; a < L.W; ++a) {
            const double2 F = row[(r.r0 + a) % Np];
            rr += wx[a] * F.x;
            ri += wx[a] * F.y;
        }
        sr += wy * rr;
        si += wy * ri;
    }
    acc[k] = make_double2(acc[k].x + wz * sr, acc[k].y + wz * si);
}

// Algorithm 6 step 5: x exp(-2 pi i w (n0 - 1)); folded visibilities conjugated.
__global__ void finish_degrid64_kernel(const VisRec64 *__restrict__ rec, int64_t M, double2 *__restrict__ vis) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M) return;
    const VisRec64 r = rec[k];
    if (r.t0 < 0) {
        vis[k] = make_double2(0.0, 0.0);
        return;
    }
    const double2 a = vis[k];
    double2 out = make_double2(a.x * r.pre_re + a.y * r.pre_im, a.y * r.pre_re - a.x * r.pre_im);
    if (r.folded) out.y = -out.y;
    vis[k] = out;
}

inline unsigned blocks64(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Both passes of the 2-D transform of one plane: rows, then columns.
cudaError_t plane_fft64(const ws_plan_s *p, double2 *plane, bool inverse, cudaStream_t s) {
    const int Np = p->L.Np;
    const size_t smem = (size_t)Np * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(fft64_lines_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fft64_lines_kernel<<<Np, 256, smem, s>>>(plane, Np, p->fft64_log, (size_t)Np, 1, p->d_tw64, inverse ? 1 : 0);
    fft64_lines_kernel<<<Np, 256, smem, s>>>(plane, Np, p->fft64_log, 1, (size_t)Np, p->d_tw64, inverse ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace

size_t fp64_record_bytes() { return sizeof(VisRec64); }

ws_status enqueue_grid64(ws_plan_s *p, const double *uvw, const double2 *vis, int64_t M, double2 *dirty,
                         cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(p->d_drop, 0, kCounters * sizeof(unsigned long long), s);
    const int64_t n_img = (int64_t)p->L.N * p->L.N;
    VisRec64 *rec = reinterpret_cast<VisRec64 *>(p->d_rec64);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_acc64, 0, (size_t)n_img * sizeof(double2), s);
    if (e == cudaSuccess && M > 0) {
        prep64_kernel<<<blocks64(M, 256), 256, 0, s>>>(p->L, uvw, M, rec, p->d_drop);
        e = cudaGetLastError();
    }
    for (int pl = 0; pl < p->L.Nw && e == cudaSuccess; ++pl) {
        e = cudaMemsetAsync(p->d_plane64, 0, (size_t)p->L.Np * p->L.Np * sizeof(double2), s);
        if (e == cudaSuccess && M > 0) {
            spread64_kernel<<<blocks64(M, 128), 128, 0, s>>>(p->L, p->d_cheb64, p->fit.degree, rec, vis, M, pl,
                                                              p->d_plane64);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = plane_fft64(p, p->d_plane64, true, s);
        if (e == cudaSuccess) {
            crop_acc64_kernel<<<blocks64(n_img, 256), 256, 0, s>>>(p->L, p->d_plane64, p->d_z64,
                                                                    (double)(pl + p->L.t_lo), p->d_acc64);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        finish_grid64_kernel<<<blocks64(n_img, 256), 256, 0, s>>>(n_img, p->d_corr64, p->d_acc64, p->L.fold, dirty);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? WS_OK : cuda_fail(e, "ws_grid (FP64 plan)");
}

ws_status enqueue_degrid64(ws_plan_s *p, const double2 *image, const double *uvw, int64_t M, double2 *vis,
                           cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(p->d_drop, 0, kCounters * sizeof(unsigned long long), s);
    if (M == 0) return e == cudaSuccess ? WS_OK : cuda_fail(e, "ws_degrid (FP64 plan)");
    const int64_t n_img = (int64_t)p->L.N * p->L.N;
    VisRec64 *rec = reinterpret_cast<VisRec64 *>(p->d_rec64);
    if (e == cudaSuccess) e = cudaMemsetAsync(vis, 0, (size_t)M * sizeof(double2), s);
    if (e == cudaSuccess) {
        prep64_kernel<<<blocks64(M, 256), 256, 0, s>>>(p->L, uvw, M, rec, p->d_drop);
        e = cudaGetLastError();
    }
    for (int pl = 0; pl < p->L.Nw && e == cudaSuccess; ++pl) {
        e = cudaMemsetAsync(p->d_plane64, 0, (size_t)p->L.Np * p->L.Np * sizeof(double2), s);
        if (e == cudaSuccess) {
            pad_screen64_kernel<<<blocks64(n_img, 256), 256, 0, s>>>(p->L, p->d_corr64, image, p->d_z64,
                                                                      (double)(pl + p->L.t_lo), p->d_plane64);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = plane_fft64(p, p->d_plane64, false, s);
        if (e == cudaSuccess) {
            gather64_kernel<<<blocks64(M, 128), 128, 0, s>>>(p->L, p->d_cheb64, p->fit.degree, rec, M, pl,
                                                              p->d_plane64, vis);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        finish_degrid64_kernel<<<blocks64(M, 256), 256, 0, s>>>(rec, M, vis);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? WS_OK : cuda_fail(e, "ws_degrid (FP64 plan)");
}

}  // namespace ws
