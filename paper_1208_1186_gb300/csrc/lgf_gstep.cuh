// One site of the gauge step on G (gauge representation, Sec. 2.1 with the
// Fourier-accelerated gradient of Sec. 2.2): from the packed accelerated
// gradient c0..c3 (Delta~_01, Delta~_02, Delta~_12, i Im Delta~_00 + Im
// Delta~_11), g = reunitarised (1 + h Delta~) with h = alpha / 2 (or the
// reunitarised exact exponential, see gstep_g), and
// G(x) <- reunitarised g G(x).  Shared by the stand-alone G update and the
// kernel that fuses it with the inverse x-y transform.
#pragma once

#include "lgf_common.cuh"

namespace lgf {

// G(x) in storage precision (row 3 completed for the 12-real form)
template <class T, int NC>
__device__ __forceinline__ M3<T> gstep_load_G(const cx<T>* G, int64_t V, int64_t s) {
  M3<T> Gt;
#pragma unroll
  for (int c = 0; c < NC; ++c) Gt.e[c / 3][c % 3] = G[c * V + s];
  if (NC == 6) complete_row3(Gt);
  return Gt;
}

// g = reunitarised (1 + h Delta~) in RT; with exact, reunitarised
// exp(h Delta~) (expm_taylor)
template <class RT, class T>
__device__ __forceinline__ M3<RT> gstep_g(cx<T> d0, cx<T> d1, cx<T> d2, cx<T> d3, RT h, bool exact = false) {
  const cx<RT> c0 = cvt<RT>(d0), c1 = cvt<RT>(d1), c2 = cvt<RT>(d2), c3 = cvt<RT>(d3);
  if (exact) {
    M3<RT> e = expm_taylor(unpack_ah(c0, c1, c2, c3, h));
    reunitarize(e);
    return e;
  }
  M3<RT> g;
  g.e[0][0] = mk<RT>(1, h * c3.re);
  g.e[0][1] = scale(c0, h);
  g.e[0][2] = scale(c1, h);
  g.e[1][0] = mk<RT>(-h * c0.re, h * c0.im);
  g.e[1][1] = mk<RT>(1, h * c3.im);
  g.e[1][2] = scale(c2, h);
  reunitarize(g);
  return g;
}

// G(x) <- reunitarised g Gt, Gt the loaded G(x)
template <class T, int NC, class RT>
__device__ __forceinline__ void gstep_store(const M3<RT>& g, const M3<T>& Gt, cx<T>* G, int64_t V, int64_t s) {
  M3<RT> Gx, r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Gx.e[i][j] = cvt<RT>(Gt.e[i][j]);
  mm<RT, 2>(r, g, Gx);
  reunitarize(r);
#pragma unroll
  for (int c = 0; c < NC; ++c) G[c * V + s] = cvt<T>(r.e[c / 3][c % 3]);
}

// RT: arithmetic of g, the product and both projections.  g_out (if not
// null) receives g; G (if not null) is updated in place.
template <class T, int NC, class RT>
__device__ __forceinline__ void gstep_site(cx<T> d0, cx<T> d1, cx<T> d2, cx<T> d3, RT h, cx<T>* G,
                                           cx<T>* __restrict__ g_out, int64_t V, int64_t s, bool exact = false) {
  const M3<RT> g = gstep_g<RT>(d0, d1, d2, d3, h, exact);
  if (g_out != nullptr) {
#pragma unroll
    for (int c = 0; c < NC; ++c) g_out[c * V + s] = cvt<T>(g.e[c / 3][c % 3]);
  }
  if (G == nullptr) return;
  gstep_store<T, NC, RT>(g, gstep_load_G<T, NC>(G, V, s), G, V, s);
}

}  // namespace lgf
