// Compile-time velocity sets of the three lattices the library instantiates.
//
// D1Q3 is given in App. A (Eq. (D1Q3lattice)); D2Q9 and D3Q19 are the
// standard sets the paper's any-dimension formulas are applied to.  Order:
// the rest velocity first, then the moving velocities in lexicographic order
// of (v_x, v_y, v_z) over {-1, 0, 1}^D (D3Q19: those with |v|^2 <= 2).  The
// set is symmetric under v -> -v and lexicographic order reverses under it,
// so opp(q) = Q - q for q > 0.  All accessors are constexpr so that, inside
// fully unrolled loops, every component and weight folds into the code.
//
// wf(q): the weights in single precision, for the float arithmetic of the
// fast paths.  The nearest floats to 4/9, 1/9, 1/36 (and 2/3, 1/6; 1/3,
// 1/18, 1/36) sum to 1 + 7.5e-9 (D2Q9; 3.0e-8 D1Q3, 1.5e-8 D3Q19), and every
// collision scales the zeroth moment of an equilibrium by that sum: the
// alpha schemes relax toward (1 + delta) times their deviation, a drift that
// grows linearly with the step count (7e-5 in alpha_g after the 2D box's
// 20,000 steps).  wf(q) are floats within 1.3e-7 (relative) of the weights
// whose exact sum is 1: the moving weights are rounded to a grid coarse
// enough that the rest weight 1 - sum(moving) is itself a float.
//
// af(q): the first-order coefficients w_q / cs2 in single precision.  The
// equilibrium's first moment is sum_q v_q af(q) (v_q . u) = u sum_q af(q) v_x^2,
// and every collision scales the momentum by that sum; 1/3 is not a binary
// fraction, so no float weights make 3 sum w v_x^2 = 1, and the momentum
// would drift like the mass above.  af(q) are floats within 6e-8 of 3 w_q
// with sum_q af(q) v_x^2 = 1 exactly.
#pragma once

namespace lbm {

constexpr double CS2 = 1.0 / 3.0;

template <int LAT> struct Lattice;

template <> struct Lattice<1> {
  static constexpr int D = 1, Q = 3;
  __host__ __device__ static constexpr int v(int q, int a) { return a != 0 ? 0 : (q == 1 ? -1 : (q == 2 ? 1 : 0)); }
  __host__ __device__ static constexpr double w(int q) { return q == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
  // 11184811 / 2^24 + 2 * 5592405 / 2^25 = 1
  __host__ __device__ static constexpr float wf(int q) {
    return q == 0 ? 11184811.0f / 16777216.0f : 5592405.0f / 33554432.0f;
  }
  // 2 * 1/2 = 1
  __host__ __device__ static constexpr float af(int q) { return q == 0 ? 0.0f : 0.5f; }
  __host__ __device__ static constexpr int opp(int q) { return q == 0 ? 0 : Q - q; }
};

template <> struct Lattice<2> {
  static constexpr int D = 2, Q = 9;
  // q = 1..8 -> cell k of the 3x3 stencil without its centre (k = 4)
  __host__ __device__ static constexpr int cell(int q) { return q == 0 ? 4 : (q <= 4 ? q - 1 : q); }
  __host__ __device__ static constexpr int v(int q, int a) {
    return a == 0 ? cell(q) / 3 - 1 : (a == 1 ? cell(q) % 3 - 1 : 0);
  }
  __host__ __device__ static constexpr double w(int q) {
    return q == 0 ? 4.0 / 9.0 : ((v(q, 0) != 0 && v(q, 1) != 0) ? 1.0 / 36.0 : 1.0 / 9.0);
  }
  // 14913081 / 2^25 + 4 * 14913081 / 2^27 + 4 * 3728270 / 2^27 = 1
  __host__ __device__ static constexpr float wf(int q) {
    return q == 0 ? 14913081.0f / 33554432.0f
                  : ((v(q, 0) != 0 && v(q, 1) != 0) ? 3728270.0f / 134217728.0f : 14913081.0f / 134217728.0f);
  }
  // 2 * 11184811 / 2^25 + 4 * 11184810 / 2^27 = 1
  __host__ __device__ static constexpr float af(int q) {
    return q == 0 ? 0.0f
                  : ((v(q, 0) != 0 && v(q, 1) != 0) ? 11184810.0f / 134217728.0f : 11184811.0f / 33554432.0f);
  }
  __host__ __device__ static constexpr int opp(int q) { return q == 0 ? 0 : Q - q; }
};

template <> struct Lattice<3> {
  static constexpr int D = 3, Q = 19;
  // q = 1..18 -> cell k = 9(v_x+1) + 3(v_y+1) + (v_z+1) of the 3x3x3 stencil,
  // the 18 cells with 1 <= |v|^2 <= 2 in increasing order
  __host__ __device__ static constexpr int cell(int q) {
    return q == 0 ? 13
         : (q <= 5 ? (q == 1 ? 1 : (q == 2 ? 3 : (q == 3 ? 4 : (q == 4 ? 5 : 7))))
         : (q <= 13 ? (q == 6 ? 9 : (q == 7 ? 10 : (q == 8 ? 11 : (q == 9 ? 12 : (q == 10 ? 14 : (q == 11 ? 15 : (q == 12 ? 16 : 17)))))))
                    : (q == 14 ? 19 : (q == 15 ? 21 : (q == 16 ? 22 : (q == 17 ? 23 : 25))))));
  }
  __host__ __device__ static constexpr int v(int q, int a) {
    return a == 0 ? cell(q) / 9 - 1 : (a == 1 ? (cell(q) / 3) % 3 - 1 : cell(q) % 3 - 1);
  }
  __host__ __device__ static constexpr double w(int q) {
    return q == 0 ? 1.0 / 3.0
                  : ((v(q, 0) * v(q, 0) + v(q, 1) * v(q, 1) + v(q, 2) * v(q, 2)) == 2 ? 1.0 / 36.0 : 1.0 / 18.0);
  }
  // 2796203 / 2^23 + 6 * 14913081 / 2^28 + 12 * 14913079 / 2^29 = 1
  __host__ __device__ static constexpr float wf(int q) {
    return q == 0 ? 2796203.0f / 8388608.0f
                  : ((v(q, 0) * v(q, 0) + v(q, 1) * v(q, 1) + v(q, 2) * v(q, 2)) == 2 ? 14913079.0f / 536870912.0f
                                                                                       : 14913081.0f / 268435456.0f);
  }
  // 2 * 5592405 / 2^25 + 8 * 11184811 / 2^27 = 1
  __host__ __device__ static constexpr float af(int q) {
    return q == 0 ? 0.0f
                  : ((v(q, 0) * v(q, 0) + v(q, 1) * v(q, 1) + v(q, 2) * v(q, 2)) == 2 ? 11184811.0f / 134217728.0f
                                                                                       : 5592405.0f / 33554432.0f);
  }
  __host__ __device__ static constexpr int opp(int q) { return q == 0 ? 0 : Q - q; }
};

// Weights and first-order coefficients in the arithmetic type R of a kernel:
// wf / af for float, w / 3 w for double.
template <class L, class R> struct WeightR;
template <class L> struct WeightR<L, float> {
  __host__ __device__ static constexpr float w(int q) { return L::wf(q); }
  __host__ __device__ static constexpr float a(int q) { return L::af(q); }
};
template <class L> struct WeightR<L, double> {
  __host__ __device__ static constexpr double w(int q) { return L::w(q); }
  __host__ __device__ static constexpr double a(int q) { return 3.0 * L::w(q); }
};
template <class L, class R> __host__ __device__ constexpr R wq(int q) { return WeightR<L, R>::w(q); }
template <class L, class R> __host__ __device__ constexpr R aq(int q) { return WeightR<L, R>::a(q); }

}  // namespace lbm
