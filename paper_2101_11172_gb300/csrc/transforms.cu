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
namespace {
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
EncodeTiled encode_tiled() {
    static const EncodeTiled fn = []() -> EncodeTiled {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiled>(f);
    }();
    return fn;
}
}  // namespace

// Element (S, R) of plane p sits at float offset 2 (((R / 4) N' + S) 4 + R % 4)
// + 2 N'^2 p: dimension 0 runs over the 8 floats of a block row, 1 over the
// N' rows S (32 bytes apart), 2 over the N'/4 column blocks (32 N' bytes
// apart), 3 over the P planes.  A box {8, 1, B, 1}, B = min(256, N'/4), is B
// column blocks of one row: 4B consecutive columns, 32B contiguous bytes in
// shared memory in column order.
cudaError_t row_tensor_map(const ws_plan_s *p, CUtensorMap *map) {
    const EncodeTiled encode = encode_tiled();
    if (!encode) return cudaErrorNotSupported;
    const cuuint64_t Np = (cuuint64_t)p->L.Np;
    const cuuint64_t dims[4] = {2 * CB, Np, Np / CB, (cuuint64_t)p->P};
    const cuuint64_t strides[3] = {2 * CB * sizeof(float), Np * 2 * CB * sizeof(float), Np * Np * sizeof(float2)};
    const cuuint32_t box[4] = {2 * CB, 1, (cuuint32_t)std::min<cuuint64_t>(256, Np / CB), 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p->d_stack, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

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
