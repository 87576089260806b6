// k_fwd.cu -- K1 launchers for ONE (input type, task kind): the analytic
// signal (Eq. 3) on the FFT engines of fft.cuh, fused with the unit-phasor
// normalisation (Eq. 4) and the store in the Gram's operand layout, or the
// backward recompute.  The build compiles this file once per pair, with
//   -DPLV_K1_F64=0|1     input float / double
//   -DPLV_K1_KIND=0..3   K1Kind (analytic.cuh)
// so that the many engine instantiations spread over parallel compiler runs.
#include "analytic.cuh"

#if !defined(PLV_K1_F64) || !defined(PLV_K1_KIND)
#error "k_fwd.cu is compiled with -DPLV_K1_F64=... -DPLV_K1_KIND=..."
#endif

namespace plv {
namespace {

using namespace fft;

#if PLV_K1_F64
typedef double Tin;
#else
typedef float Tin;
#endif
constexpr int KIND = PLV_K1_KIND;

template <typename T_, int K_>
struct TaskOf {
    typedef FwdTask<T_, K_> type;
    static __host__ __device__ type make(const void *x, int64_t ldx, void *P, float *, int N,
                                         int64_t ld) {
        return type{(const T_ *)x, ldx, P, N, ld};
    }
};
template <typename T_>
struct TaskOf<T_, kK1Prep> {
    typedef PrepTask<T_> type;
    static __host__ __device__ type make(const void *x, int64_t ldx, void *P, float *rinv, int N,
                                         int64_t ld) {
        return type{(const T_ *)x, ldx, (float *)P, rinv, ld, nullptr, N};
    }
};
typedef TaskOf<Tin, KIND> Tk;

// The grouped any-length launch: persistent over (problem, row pair) items
// of one thread class.  A CTA copies the problem's descriptor to shared
// memory when the problem changes (items of one problem are contiguous per
// CTA stride, so this is rare).
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 65536 / (kConvRegs * THREADS))
k_hilbert_conv_group(const K1Desc *__restrict__ descs, const int2 *__restrict__ items,
                     int64_t n) {
    extern __shared__ __align__(16) float2 smem[];
    __shared__ float s_pow;
    __shared__ __align__(16) int s_desc[sizeof(K1Desc) / 4];
    static_assert(sizeof(K1Desc) % 4 == 0, "descriptor copied as 32-bit words");
    const K1Desc &d = *reinterpret_cast<const K1Desc *>(s_desc);
    if (threadIdx.x == 0) s_pow = 0.f;
    int cur = -1;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const int2 w = __ldg(&items[i]);
        if (w.x != cur) {  // uniform: every thread reads the same item
            __syncthreads();  // the previous pair no longer reads the descriptor
            if (threadIdx.x < (int)(sizeof(K1Desc) / 4))
                s_desc[threadIdx.x] =
                    __ldg(reinterpret_cast<const int *>(descs + w.x) + threadIdx.x);
            __syncthreads();
            cur = w.x;
        }
        const auto task = Tk::make(d.x, d.ldx, d.P, nullptr, d.N, d.ld);
        conv_pair(task, d.plan, d.T, d.ld, d.rows, (int64_t)w.y, smem, &s_pow);
    }
}

template <int C>
cudaError_t launch_group_class(const Handle *h, cudaStream_t s, const K1Group &g) {
    constexpr int THREADS = conv_class_threads(C);
    auto kern = k_hilbert_conv_group<THREADS>;
    static LaunchSetup ls;
    int per_sm = 0;
    cudaError_t e = setup_once(ls, kern, THREADS, conv_smem(conv_class_max_M(C)), per_sm);
    if (e != cudaSuccess) return e;
    const int c = C;
    const int64_t n = g.count[c];
    if (n == 0) return cudaSuccess;
    if (g.per_sm[c] > 0 && g.per_sm[c] < per_sm) per_sm = g.per_sm[c];
    int64_t grid = (int64_t)per_sm * h->num_sms;
    if (grid > n) grid = n;
    kern<<<(unsigned)grid, THREADS, conv_smem(g.max_M[c]), s>>>(g.descs, g.items + g.begin[c],
                                                               n);
    return cudaGetLastError();
}

}  // namespace

template <typename Tin_, int KIND_>
cudaError_t k1_pow2(const Handle *h, cudaStream_t s, const K1Args &a) {
    if constexpr (KIND_ == kK1Prep) {
        if (a.Ps) {  // the backward recompute, with the split operand as well
            const PrepTask<Tin_, true> task{(const Tin_ *)a.x, a.ldx, (float *)a.P, a.rinv, a.ld,
                                            a.Ps, a.N};
            return launch_hilbert_pow2(h->num_sms, s, a.log2T, task, twiddle_table(h, a.log2T),
                                       a.rows);
        }
    }
    const auto task = TaskOf<Tin_, KIND_>::make(a.x, a.ldx, a.P, a.rinv, a.N, a.ld);
    return launch_hilbert_pow2(h->num_sms, s, a.log2T, task, twiddle_table(h, a.log2T), a.rows);
}

template <typename Tin_, int KIND_>
cudaError_t k1_conv(const Handle *h, cudaStream_t s, const K1Args &a, const ConvPlan &plan) {
    if constexpr (KIND_ == kK1Prep) {
        if (a.Ps) {
            const PrepTask<Tin_, true> task{(const Tin_ *)a.x, a.ldx, (float *)a.P, a.rinv, a.ld,
                                            a.Ps, a.N};
            return launch_hilbert_conv(h->num_sms, s, task, plan, a.T, a.ld, a.rows);
        }
    }
    const auto task = TaskOf<Tin_, KIND_>::make(a.x, a.ldx, a.P, a.rinv, a.N, a.ld);
    return launch_hilbert_conv(h->num_sms, s, task, plan, a.T, a.ld, a.rows);
}

template <typename Tin_, int KIND_>
cudaError_t k1_conv_group(const Handle *h, cudaStream_t s, const K1Group &g) {
    if constexpr (KIND_ == kK1Prep) {
        return cudaErrorInvalidValue;  // the backward recompute is not grouped
    } else {
        static_assert(kConvClasses == 4, "one launch per class");
        cudaError_t e = launch_group_class<0>(h, s, g);
        if (e == cudaSuccess) e = launch_group_class<1>(h, s, g);
        if (e == cudaSuccess) e = launch_group_class<2>(h, s, g);
        if (e == cudaSuccess) e = launch_group_class<3>(h, s, g);
        return e;
    }
}

template cudaError_t k1_pow2<Tin, KIND>(const Handle *, cudaStream_t, const K1Args &);
template cudaError_t k1_conv<Tin, KIND>(const Handle *, cudaStream_t, const K1Args &,
                                        const ConvPlan &);
template cudaError_t k1_conv_group<Tin, KIND>(const Handle *, cudaStream_t, const K1Group &);

}  // namespace plv
