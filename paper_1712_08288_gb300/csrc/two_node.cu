// two_node.cu -- the two-node variant of the boundary scheme (Sec. 2, Remark (2),
// Eq. 2.11) on top of the fused sweep.
//
// Eq. 2.10 approximates f_ibar(x_f, t+1) by f_ibar(x_f, t) (Eq. 2.9).  When the node
// x_l = x_f + e_i behind the boundary node is fluid, the exact value is the
// post-collision f'_ibar(x_l, t), which streams to x_f.  The two schemes differ by
//   v_2node - v_1node = b A (f'_ibar(x_l, t) - f_ibar(x_f, t)),
// with A = (1 + l - 2 gamma)/(1 + l) (b A is the coefficient the sweep already
// uses).  Both terms are known before the step, so a pre-pass over the links
// computes the difference (colliding x_l's populations with the sweep's own
// collision), the unchanged sweep writes the single-node value, and a post-pass adds
// the difference where the value now sits: the link buffer after an even step, the
// node's own slot i after an odd one.
#include "sweep.cuh"

namespace lbm {

namespace {

constexpr int kTnThreads = 128;

template <class L, class T>
__global__ void two_node_pre_kernel(const SweepArgs<typename Storage<T>::C> sa, AuxArgs a,
                                    bool odd, const TwoNodeLink *__restrict__ tn, long long n_tn,
                                    typename Storage<T>::C *__restrict__ delta) {
  using C = typename Storage<T>::C;
  constexpr int Q = L::Q;
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= n_tn) return;
  const TwoNodeLink e = tn[j];
  C g[Q], gp[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) g[q] = C(Storage<T>::load(population_address<L, T>(q, e.xl, odd, a)));
  C drho;
  collide<L, C>(g, gp, sa, drho);
  // gp[d] for the runtime direction d, without a local-memory table
  C fl_next = C(0);
#pragma unroll
  for (int q = 1; q < Q; ++q)
    if (q == e.d) fl_next = gp[q];
  const C fd = C(Storage<T>::load(population_address<L, T>(e.d, e.xf, odd, a)));
  const LinkCoef<C> *coef = static_cast<const LinkCoef<C> *>(sa.geo.coef);
  delta[j] = coef[e.k].a * (fl_next - fd);
}

template <class L, class T>
__global__ void two_node_post_kernel(AuxArgs a, bool next_odd, const TwoNodeLink *__restrict__ tn,
                                     long long n_tn, const typename Storage<T>::C *__restrict__ delta) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= n_tn) return;
  const TwoNodeLink e = tn[j];
  T *p = next_odd ? static_cast<T *>(const_cast<void *>(a.lnk)) + e.k
                  : static_cast<T *>(a.pop) + (long long)L::opp_rt(e.d) * a.S + e.xf;
  Storage<T>::store(p, Storage<T>::load(p) + delta[j]);
}

unsigned tn_blocks(long long n) { return (unsigned)((n + kTnThreads - 1) / kTnThreads); }

}  // namespace

cudaError_t launch_two_node(int lattice, int precision, const SweepArgs<double> &a64,
                            const SweepArgs<float> &a32, const AuxArgs &a, bool odd, bool post,
                            const TwoNodeLink *tn, long long n_tn, void *delta, cudaStream_t st) {
  if (n_tn <= 0) return cudaSuccess;
  return with_lattice(lattice, [&](auto lat) {
    using L = decltype(lat);
    return with_storage(precision, [&](auto *tp) {
      using T = std::remove_pointer_t<decltype(tp)>;
      using C = typename Storage<T>::C;
      const SweepArgs<C> *sa;
      if constexpr (sizeof(C) == 8) sa = &a64;
      else sa = &a32;
      if (!post)
        two_node_pre_kernel<L, T><<<tn_blocks(n_tn), kTnThreads, 0, st>>>(*sa, a, odd, tn, n_tn,
                                                                          static_cast<C *>(delta));
      else
        two_node_post_kernel<L, T><<<tn_blocks(n_tn), kTnThreads, 0, st>>>(
            a, !odd, tn, n_tn, static_cast<const C *>(delta));
      return cudaGetLastError();
    });
  });
}

}  // namespace lbm
