// k_aos.cu -- host side of the AOS step of Eq. 4: tensor maps for the
// column strips, kernel configuration and dispatch to the solver variant
// whose compile-time chunk length fits the line (see aos_solver.cuh; the
// variants are instantiated in k_aos_v*.cu so they compile in parallel).
#include <cudaTypedefs.h>
#include <dlfcn.h>

#include "aos_solver.cuh"

namespace kz {
namespace aos {
KZ_AOS_VARIANTS(KZ_AOS_DECLARE)
}  // namespace aos

namespace {

constexpr size_t kSmemBudget = 220 * 1024;
int g_cols_pref = 16;  // widest column strip tried first

size_t row_smem(int w)
{
    const int m = aos::chunk_len(w);
    if (m == 0) return 0;
    const int P = 32 * aos::warps_per_line(w);
    const int rows = 4 / aos::warps_per_line(w);
    return (size_t)rows * (2 * aos::row_stride_floats(P, m) + 8 * P) * sizeof(float);
}

size_t cols_smem(int h, int cols)
{
    const int m = aos::chunk_len(h);
    if (m == 0) return 0;
    const int P = 32 * aos::warps_per_line(h);
    return ((size_t)2 * aos::rows_staged(P, m) * cols + (size_t)8 * cols * P) * sizeof(float);
}

int cols_per_cta(int h)
{
    if (aos::chunk_len(h) == 0) return 0;
    if (g_cols_pref == 16 && cols_smem(h, 16) <= kSmemBudget) return 16;
    if (cols_smem(h, 8) <= kSmemBudget) return 8;
    if (cols_smem(h, 4) <= kSmemBudget) return 4;
    return 0;
}

const char* g_encode_err = "";

// cuTensorMapEncodeTiled from the driver: through the runtime's entry-point
// query, else straight from libcuda.so.1 (no link-time driver dependency).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn) return fn;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e == cudaSuccess && q == cudaDriverEntryPointSuccess && p) {
        fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        return fn;
    }
    void* lib = dlopen("libcuda.so.1", RTLD_NOW | RTLD_NOLOAD);
    if (!lib) lib = dlopen("libcuda.so.1", RTLD_NOW);
    if (lib) p = dlsym(lib, "cuTensorMapEncodeTiled");
    if (p) {
        fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        return fn;
    }
    g_encode_err = e != cudaSuccess ? "cudaGetDriverEntryPointByVersion failed and libcuda.so.1 has no cuTensorMapEncodeTiled"
                                    : "cuTensorMapEncodeTiled not found in the driver";
    return nullptr;
}

}  // namespace

bool make_plane_map(CUtensorMap* map, const float* base, int pitch, int w, int h, int box_x, int box_y)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)h};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
    cuuint32_t estr[2] = {1u, 1u};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

namespace {
// 2-D map of a w x h FP32 plane with the given pitch, box COLS x 256.
bool make_strip_map(CUtensorMap* map, const float* base, int pitch, int w, int h, int cols)
{
    return make_plane_map(map, base, pitch, w, h, cols, 256);
}
}  // namespace

const char* aos_config_error() { return g_encode_err; }

cudaError_t configure_aos_kernels()
{
    cudaError_t e = cudaSuccess;
#define KZ_CFG(M, NW) \
    if (e == cudaSuccess) e = aos::configure_m<M, NW>();
    KZ_AOS_VARIANTS(KZ_CFG)
#undef KZ_CFG
    if (e == cudaSuccess && !encode_fn()) e = cudaErrorNotSupported;
    return e;
}

size_t aos_rows_smem_bytes(int w)
{
    const size_t b = row_smem(w);
    return b <= kSmemBudget ? b : 0;
}

size_t aos_cols_smem_bytes(int h)
{
    const int c = cols_per_cta(h);
    return c == 0 ? 0 : cols_smem(h, c);
}

cudaError_t launch_aos_rows(const float* L, const float* g, float* ux, float* acc, int pitch, int w, int h,
                            float tau, int* d_status, cudaStream_t st)
{
    const size_t smem = aos_rows_smem_bytes(w);
    if (smem == 0) return cudaErrorInvalidValue;
    if (acc && ((pitch & 3) != 0 || ((uintptr_t)acc & 15) != 0)) return cudaErrorInvalidValue;
    const int nw = aos::warps_per_line(w), m = aos::chunk_len(w);
    const aos::RowsArgs args{L, g, ux, acc, pitch, w, h, tau, d_status, smem, st};
#define KZ_ROWS(M, NW) \
    if (nw == NW && m == M) return aos::launch_rows_m<M, NW>(args);
    KZ_AOS_VARIANTS(KZ_ROWS)
#undef KZ_ROWS
    return cudaErrorInvalidValue;
}

cudaError_t launch_aos_cols(const float* L, const float* g, const float* ux, float* Lnext, int pitch, int w, int h,
                            float tau, int* d_status, cudaStream_t st, int cols)
{
    const int c = cols == 0 ? cols_per_cta(h) : cols;
    if (c == 0 || (c != 4 && c != 8 && c != 16) || cols_smem(h, c) > kSmemBudget) return cudaErrorInvalidValue;
    aos::ColsArgs args;
    if (!make_strip_map(&args.mL, L, pitch, w, h, c) || !make_strip_map(&args.mG, g, pitch, w, h, c))
        return cudaErrorInvalidValue;
    if (!ux && ((pitch & 3) != 0 || ((uintptr_t)Lnext & 15) != 0)) return cudaErrorInvalidValue;
    args.g = g;
    args.ux = ux;
    args.Lnext = Lnext;
    args.pitch = pitch;
    args.w = w;
    args.h = h;
    args.tau = tau;
    args.status = d_status;
    args.smem = cols_smem(h, c);
    args.cols = c;
    args.st = st;
    const int nw = aos::warps_per_line(h), m = aos::chunk_len(h);
#define KZ_COLS(M, NW) \
    if (nw == NW && m == M) return aos::launch_cols_m<M, NW>(args);
    KZ_AOS_VARIANTS(KZ_COLS)
#undef KZ_COLS
    return cudaErrorInvalidValue;
}

}  // namespace kz
