// Per-bin arithmetic of the spectral solves (Sec. 3.1, Eq. 8-9) and of the
// packed column-0 bins, shared by the forward column pass and the adjoint's
// recomputation of a step.
#pragma once
#include "common.cuh"

namespace gfd {

// Bins (k, 0) and (k, N/2) of a real image's packed half spectrum, from the
// column-0 values Z[k] and Z[-k]: A = (Z[k] + conj Z[-k]) / 2,
// B = (Z[k] - conj Z[-k]) / (2i); and back, Z[k] = A + i B.
GFD_D void unpack_pair(float2 Sk, float2 Smk, float2& A, float2& Bv) {
  const float2 c = cconj(Smk);
  A = cscale(cadd(Sk, c), 0.5f);
  const float2 D = csub(Sk, c);
  Bv = make_float2(0.5f * D.y, -0.5f * D.x);  // D / (2i)
}
GFD_D float2 pack_pair(float2 A, float2 B) { return make_float2(A.x - B.y, A.y + B.x); }

// Eq. 9 (u_p) and Eq. 8 (u_I) at one bin:
//   U_p = (conj(H) Y + lam U_E) / (|H|^2 + lam)
//   U_I = (conj(H) Y + lam D2 U_E) / (|H|^2 + lam D2),  D2 = |F(nabla)|^2.
GFD_D void solve_bin(float2 U, float2 H, float2 Y, float lam, float D2, bool branch,
                     float2& UI, float2& Up) {
  if (branch) {  // lambda = inf: u_I = u_p = u_E (Sec. 3.2)
    UI = U;
    Up = U;
    return;
  }
  const float2 HY = make_float2(fmaf(H.x, Y.x, H.y * Y.y), fmaf(H.x, Y.y, -H.y * Y.x));
  const float a = fmaf(H.x, H.x, H.y * H.y);
  const float ip = __frcp_rn(a + lam);
  Up = make_float2(fmaf(lam, U.x, HY.x) * ip, fmaf(lam, U.y, HY.y) * ip);
  const float lg = lam * D2;
  const float den = a + lg;
  if (den > 0.0f) {
    const float ii = __frcp_rn(den);
    UI = make_float2(fmaf(lg, U.x, HY.x) * ii, fmaf(lg, U.y, HY.y) * ii);
  } else {
    UI = U;
  }
}

}  // namespace gfd
