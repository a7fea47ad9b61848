// Per-pixel outer-iteration steps (Sec. 2):
//  * IRLS weights  w_i = max(|(L x)_i|, eps)^(-1/2)                 (Alg. 1)
//  * MM shift      w_i = u_i (1 - (eps^2/(u_i^2 + eps^2))^(1/2)), u = L x (Eq. (wreg))
//  * SB update     d = shrink(L x + g, tau), g = g + L x - d          (Alg. 3)
//  * RC numerator / denominator ||x^(k+1) - x^(k)||^2, ||x^(k)||^2  (Eq. (stop))
// fused into one pass that also forms x^(k+1) = x^(k) + delta.
#pragma once
#include "lsqr.cuh"

namespace db {

template <typename Acc> __device__ __forceinline__ Acc irls_w(Acc q, Acc eps) {
  Acc a = fabs(q);
  a = a > eps ? a : eps;
  return Acc(1) / sqrt(a);
}
template <typename Acc> __device__ __forceinline__ Acc mm_c(Acc u, Acc eps) {
  return u * (Acc(1) - sqrt(eps * eps / (u * u + eps * eps)));
}
template <typename Acc> __device__ __forceinline__ Acc shrink(Acc x, Acc tau) {
  Acc a = fabs(x) - tau;
  a = a > Acc(0) ? a : Acc(0);
  return x > Acc(0) ? a : (x < Acc(0) ? -a : Acc(0));
}

enum AuxMode { AUX_APPROACH_I = 0, AUX_FROM_X = 1 };

// Initial auxiliaries of a level (Sec. 4.1).
template <typename T>
__global__ void k_aux_init(int m, int solver, int mode, const typename Traits<T>::X* __restrict__ x, T* a0x,
                           T* a0y, T* a1x, T* a1y, double eps_irls, double eps_mm, double tau) {
  using Acc = typename Traits<T>::Acc;
  size_t n = (size_t)m * m;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(i % m), c = (int)(i / m);
    const bool vx = r < m - 1, vy = c < m - 1;
    Acc qx = 0, qy = 0;
    if (mode == AUX_FROM_X) {
      Acc xv = to_acc(x[i]);
      if (vx) qx = to_acc(x[i + 1]) - xv;
      if (vy) qy = to_acc(x[i + m]) - xv;
    }
    Acc ox = 0, oy = 0, gx = 0, gy = 0;
    if (solver == 0) {
      if (mode == AUX_APPROACH_I) { ox = vx ? Acc(1) : Acc(0); oy = vy ? Acc(1) : Acc(0); }
      else { ox = vx ? irls_w<Acc>(qx, (Acc)eps_irls) : Acc(0); oy = vy ? irls_w<Acc>(qy, (Acc)eps_irls) : Acc(0); }
    } else if (solver == 1) {
      if (mode == AUX_FROM_X) { ox = mm_c<Acc>(qx, (Acc)eps_mm); oy = mm_c<Acc>(qy, (Acc)eps_mm); }
    } else {
      if (mode == AUX_FROM_X) {   // one shrinkage step from g = 0
        ox = shrink<Acc>(qx, (Acc)tau); oy = shrink<Acc>(qy, (Acc)tau);
        gx = qx - ox; gy = qy - oy;
      }
      a1x[i] = store_cast<T, Acc>(gx);
      a1y[i] = store_cast<T, Acc>(gy);
    }
    a0x[i] = store_cast<T, Acc>(ox);
    a0y[i] = store_cast<T, Acc>(oy);
  }
}

// x_new = (warm ? x_old : 0) + dlt; auxiliaries for the next outer iteration
// from L x_new; partial sums of ||x_new - x_old||^2 and ||x_old||^2 reduced
// by the last block into out[0..1]. solver < 0 skips the auxiliary update.
template <typename T>
__global__ void __launch_bounds__(256) k_outer_update(int m, int solver, int warm,
    const typename Traits<T>::X* __restrict__ x_old, const typename Traits<T>::X* __restrict__ dlt,
    typename Traits<T>::X* __restrict__ x_new,
    T* a0x, T* a0y, T* a1x, T* a1y, double eps_irls, double eps_mm, double tau,
    double* part, unsigned* cnt, double* out) {
  using Acc = typename Traits<T>::Acc;
  using X = typename Traits<T>::X;
  __shared__ double scratch[2 * 32];
  __shared__ int s_flag;
  size_t n = (size_t)m * m;
  double red[2] = {0.0, 0.0};
  Acc s0 = 0, s1 = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    int r = (int)(i % m), c = (int)(i / m);
    auto xn_at = [&](size_t k) -> Acc {
      return (warm ? to_acc(x_old[k]) : Acc(0)) + to_acc(dlt[k]);
    };
    const Acc xo = to_acc(x_old[i]);
    const Acc xn = xn_at(i);
    x_new[i] = store_cast<X, Acc>(xn);
    const Acc dx = xn - xo;
    s0 += dx * dx;
    s1 += xo * xo;
    const bool vx = r < m - 1, vy = c < m - 1;
    const Acc qx = vx ? xn_at(i + 1) - xn : Acc(0);
    const Acc qy = vy ? xn_at(i + m) - xn : Acc(0);
    if (solver < 0) {
      // no auxiliary update (plain x_new = x_old + delta)
    } else if (solver == 0) {
      a0x[i] = store_cast<T, Acc>(vx ? irls_w<Acc>(qx, (Acc)eps_irls) : Acc(0));
      a0y[i] = store_cast<T, Acc>(vy ? irls_w<Acc>(qy, (Acc)eps_irls) : Acc(0));
    } else if (solver == 1) {
      a0x[i] = store_cast<T, Acc>(mm_c<Acc>(qx, (Acc)eps_mm));
      a0y[i] = store_cast<T, Acc>(mm_c<Acc>(qy, (Acc)eps_mm));
    } else {
      const Acc gx = to_acc(a1x[i]), gy = to_acc(a1y[i]);
      const Acc dx2 = shrink<Acc>(qx + gx, (Acc)tau), dy2 = shrink<Acc>(qy + gy, (Acc)tau);
      a0x[i] = store_cast<T, Acc>(dx2);
      a0y[i] = store_cast<T, Acc>(dy2);
      a1x[i] = store_cast<T, Acc>(gx + qx - dx2);
      a1y[i] = store_cast<T, Acc>(gy + qy - dy2);
    }
  }
  red[0] = (double)s0;
  red[1] = (double)s1;
  block_sum<2>(red, scratch);
  if (threadIdx.x == 0) {
    part[blockIdx.x * 2] = red[0];
    part[blockIdx.x * 2 + 1] = red[1];
    __threadfence();
    unsigned old = atomicAdd(cnt, 1u);
    s_flag = (old == gridDim.x - 1);
    __threadfence();
  }
  __syncthreads();
  if (s_flag && threadIdx.x < 32) {
    double t0 = 0, t1 = 0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += 32) {
      t0 += __ldcg(part + 2 * b);
      t1 += __ldcg(part + 2 * b + 1);
    }
    t0 = warp_sum(t0);
    t1 = warp_sum(t1);
    if (threadIdx.x == 0) { out[0] = t0; out[1] = t1; *cnt = 0; }
  }
}

// Generic fixed-order sum of squares / dot products of two Acc vectors into
// out (double), with the same last-block pattern.
template <typename A1, typename A2>
__global__ void __launch_bounds__(256) k_dot(size_t n, const A1* __restrict__ x, const A2* __restrict__ y,
                                             double* part, unsigned* cnt, double* out) {
  __shared__ double scratch[32];
  __shared__ int s_flag;
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc += (double)to_acc(x[i]) * (double)to_acc(y[i]);
  double red[1] = {acc};
  block_sum<1>(red, scratch);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = red[0];
    __threadfence();
    unsigned old = atomicAdd(cnt, 1u);
    s_flag = (old == gridDim.x - 1);
    __threadfence();
  }
  __syncthreads();
  if (s_flag && threadIdx.x < 32) {
    double t = 0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += 32) t += __ldcg(part + b);
    t = warp_sum(t);
    if (threadIdx.x == 0) { *out = t; *cnt = 0; }
  }
}

}  // namespace db
