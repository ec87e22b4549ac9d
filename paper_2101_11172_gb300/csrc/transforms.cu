// Fused plane transforms of the improved W-stacking method (sm_103a).
//
// Degridding (Algorithm 6 steps 3a-3c) for plane t:
//   Q_t = pad_{N'}( g exp(-2 pi i t z) ),  g = h_x h_y h_z f   (image, N x N)
//   F_t[S][R] = sum_{I,J} Q_t[I][J] exp(-2 pi i (S I + R J) / N')
// is split into
//   fwd_rows  (screen + zero pad + DFT over J, only the N image rows I)
//   fwd_cols  (zero pad in I + DFT over I, every column R, all N' outputs S).
// Gridding (Algorithm 5 steps 3b-5) for plane t:
//   P_t[I][J] = sum_{S,R} G_t[S][R] exp(+2 pi i (S I + R J) / N'), kept on the crop
//   D[I][J]  += P_t[I][J] exp(+2 pi i t z[I][J])   (sum over t, compensated)
//   dirty     = h_x h_y h_z D
// is split into
//   inv_cols  (DFT over S of every column R, only the N crop rows I kept)
//   inv_rows  (DFT over R of each crop row, crop columns J, screen, sum over t).
// Zero padding is never stored or read (the first FFT stage produces zeros
// itself) and the crop is applied by the last stage's stores.  The
// intermediate (N crop rows x N' columns) stays in place in rows 0..N-1 of
// each column block of the plane (layout in common.cuh).
#include "transforms_impl.cuh"

namespace ws {

namespace tf {
const Ops &ops_runtime_pow2() {
    static const Ops o = ops_of<0>();
    return o;
}
const Ops &ops_runtime_mixed() {
    static const Ops o = ops_of<1>();
    return o;
}
}  // namespace tf

namespace {
// The variant for an N'-point plan: a compile-time plan when one exists.
const tf::Ops &ops_for(int Np, bool mixed) {
    switch (Np) {
        case 512: return tf::ops_512();
        case 1024: return tf::ops_1024();
        case 2048: return tf::ops_2048();
        case 4096: return tf::ops_4096();
        default: return mixed ? tf::ops_runtime_mixed() : tf::ops_runtime_pow2();
    }
}
}  // namespace

// Largest dynamic shared memory any transform kernel of this plan asks for
// (the compile-time inv_rows double buffer is checked by its own setup).
size_t transform_smem_bytes(const FftPlan &F, int N) {
    size_t b = tf::smem2(F);
    if (tf::smem_rows(F, N) > b) b = tf::smem_rows(F, N);
    if (tf::smem_fwd_rows(F, N, false) > b) b = tf::smem_fwd_rows(F, N, false);
    return b;
}

cudaError_t setup_transform_kernels(const FftPlan &F, int N) {
    return ops_for(F.n, (F.n & (F.n - 1)) != 0).setup(F, N);
}

cudaError_t launch_fwd_rows(const ws_plan_s *p, int chunk, int planes, cudaStream_t s) {
    return ops_for(p->L.Np, p->fft_mixed).fwd_rows(p, chunk, planes, s);
}

cudaError_t launch_fwd_cols(const ws_plan_s *p, int chunk, int planes, cudaStream_t s) {
    return ops_for(p->L.Np, p->fft_mixed).fwd_cols(p, chunk, planes, s);
}

cudaError_t launch_inv_cols(const ws_plan_s *p, int chunk, int planes, cudaStream_t s) {
    return ops_for(p->L.Np, p->fft_mixed).inv_cols(p, chunk, planes, s);
}

cudaError_t launch_inv_rows(const ws_plan_s *p, int chunk, int planes, bool first, bool last, float2 *dirty,
                            cudaStream_t s) {
    return ops_for(p->L.Np, p->fft_mixed).inv_rows(p, chunk, planes, first, last, dirty, s);
}

}  // namespace ws
