// rbl_erfc_fit.cuh -- generated by erfc_fit.py (do not edit): coefficients of
// erfc(x) = t h(t) exp(-x^2), t = 1 / (1 + P x), h(t) = sum_k A_k t^k, a
// least-squares fit of the relative error of h at Chebyshev nodes (max relative
// error of erfc in exact arithmetic about 1.3e-7 on [0, 10]).
#pragma once

namespace rbl {

constexpr float kErfcP = 4.000000060e-01f;
constexpr int kErfcDegree = 8;

// A_k (a function, so that unrolled device code folds each one to an immediate)
__host__ __device__ constexpr float erfc_fit_coef(int k)
{
    return k == 0 ? 2.256758660e-01f :
         k == 1 ? 2.256697714e-01f :
         k == 2 ? 2.078385800e-01f :
         k == 3 ? 1.685781777e-01f :
         k == 4 ? 1.412773430e-01f :
         k == 5 ? -5.255409982e-03f :
         k == 6 ? 1.686438620e-01f :
         k == 7 ? -1.826153398e-01f :
         k == 8 ? 5.018728971e-02f :
        0.0f;
}

} // namespace rbl
