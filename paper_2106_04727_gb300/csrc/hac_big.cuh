// GPU-wide evaluation kernels of big cluster pairs (internal): templates
// instantiated per linkage in hac_big_complete.cu and hac_big_average.cu.
#pragma once

#include "hac_impl.cuh"

#include <algorithm>

namespace {

using namespace hacg;

__device__ __forceinline__ int *bs_req(const State &s, int k) {
  return s.bsched + BS_LIST + k * (2 * BS_B + 1);
}
__device__ __forceinline__ int *bs_pre(const State &s, int k) { return bs_req(s, k) + BS_B; }

// tile `tile` of kind k: the request (index within the batch) and the
// tile's position inside it
__device__ __forceinline__ int bk_find(const State &s, int k, int tile, int &q0) {
  const int n = s.bsched[BS_META + 3 * k];
  const int *pr = bs_pre(s, k);
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pr[mid] <= tile) lo = mid;
    else hi = mid;
  }
  q0 = tile - pr[lo];
  return bs_req(s, k)[lo];
}

// the next tile of kind k for this CTA (dynamic: CTAs that finish early take
// more), or -1 when none is left
__device__ __forceinline__ int bk_next(const State &s, int k, int *sh_tile) {
  if (threadIdx.x == 0) {
    const int t = atomicAdd(&s.bsched[BS_META + 3 * k + 2], 1);
    *sh_tile = t < s.bsched[BS_META + 3 * k + 1] ? t : -1;
  }
  __syncthreads();
  const int t = *sh_tile;
  return t;
}

// block reduction of the tile's partial in a fixed order (deterministic)
template <int LK>
__device__ __forceinline__ void bk_store(const State &s, double v, double *red, int slot) {
  for (int o = 16; o; o >>= 1) {
    const double u = __shfl_xor_sync(0xffffffffu, v, o);
    v = LK == 0 ? fmax(v, u) : v + u;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = red[0];
    for (int w = 1; w < BIG_TPB / 32; ++w) t = LK == 0 ? fmax(t, red[w]) : t + red[w];
    s.bpart[slot] = t;
  }
}

// FP64 tiles (kind 2): 512 points of the larger cluster (two per thread)
// against the smaller one staged through shared memory.
template <int LK, int DP>
__global__ void __launch_bounds__(BIG_TPB) k_big_eval64(State s, int r0) {
  __shared__ double sh[BIG_TPB * DP];
  __shared__ double red[BIG_TPB / 32];
  __shared__ int sh_tile;
  const double *P = s.p64[s.cur];
  const int base = s.bsched[BS_META + 1] + s.bsched[BS_META + 3 + 1];  // after kinds 0, 1
  for (;;) {
    const int tile = bk_next(s, 2, &sh_tile);
    if (tile < 0) break;
    int q0;
    const int r = r0 + bk_find(s, 2, tile, q0);
    int sL = s.breq_sa[r], nL = s.breq_na[r], sS = s.breq_sb[r], nS = s.breq_nb[r];
    if (nS > nL) {
      int t0 = sL; sL = sS; sS = t0;
      t0 = nL; nL = nS; nS = t0;
    }
    const int sch = bk_chunk(2, nL, nS, s.d);
    const int ts = (nS + sch - 1) / sch;  // chunks of the smaller cluster
    const int sc0 = (q0 % ts) * sch, sc1 = min(nS, sc0 + sch);
    const int l0 = (q0 / ts) * BIG_TILE + threadIdx.x, l1 = l0 + BIG_TPB;
    const bool v0 = l0 < nL, v1 = l1 < nL;
    double x0[DP], x1[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      x0[k] = v0 ? P[(size_t)(sL + l0) * DP + k] : 0.0;
      x1[k] = v1 ? P[(size_t)(sL + l1) * DP + k] : 0.0;
    }
    double acc = 0.0, macc = 0.0;
    for (int c0 = sc0; c0 < sc1; c0 += BIG_TPB) {
      const int cn = min(BIG_TPB, sc1 - c0);
      __syncthreads();
      for (int i = threadIdx.x; i < cn * DP; i += BIG_TPB) sh[i] = P[(size_t)(sS + c0) * DP + i];
      __syncthreads();
      for (int j = 0; j < cn; ++j) {
        double d0 = 0, d1 = 0;
#pragma unroll
        for (int k = 0; k < DP; ++k) {
          const double y = sh[j * DP + k];
          const double t0 = x0[k] - y, t1 = x1[k] - y;
          d0 = d0 + t0 * t0;
          d1 = d1 + t1 * t1;
        }
        if (LK == 0) {
          if (v0) macc = fmax(macc, d0);
          if (v1) macc = fmax(macc, d1);
        } else {
          acc += (v0 ? sqrt(d0) : 0.0) + (v1 ? sqrt(d1) : 0.0);
        }
      }
    }
    bk_store<LK>(s, LK == 0 ? macc : acc, red, base + tile);
  }
}

// FP32 tiles, specialised on the true dimension D (rows have stride DP):
// PPT points of the larger cluster per thread, packed in pairs so that every
// subtract and multiply-add is one f32x2 instruction for two point pairs;
// the smaller cluster is staged through shared memory 256 points at a time,
// each coordinate duplicated into both halves of a 64-bit word.  Square
// roots use the hardware approximation (sqrt.approx.f32); with it a term's
// relative error stays within ((D+1)/2 + 4)u <= (D+16)u, the bound the search
// states for FP32 distances.  Packed operations round each half as the scalar
// instruction would.

// One staged chunk of the smaller cluster against a thread's NP point pairs.
// Average: each half of `part` takes 4 x NP terms per group of 4 staged
// points (at most 16); 16 groups are summed in FP32 before each FP64 add
// (relative error <= 30u per FP64 add, as before packing).
template <int LK, int D, int NP, bool FULL>
__device__ __forceinline__ void big32_chunk(const unsigned long long *sh, int cn,
                                            const unsigned long long (&x)[NP][D],
                                            const bool (&v)[2 * NP], double &acc, float &macc) {
  unsigned long long part2 = 0ull;  // (0.f, 0.f)
  int groups = 0;
  for (int j0 = 0; j0 < cn; j0 += 4) {
    const int jn = min(4, cn - j0);
    unsigned long long part = 0ull;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      if (jj < jn) {
        const unsigned long long *y = sh + (j0 + jj) * D;
        unsigned long long yk[D];
#pragma unroll
        for (int k = 0; k < D; ++k) yk[k] = y[k];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          unsigned long long t = f2_sub(x[q][0], yk[0]);
          unsigned long long d2 = f2_mul(t, t);
#pragma unroll
          for (int k = 1; k < D; ++k) {
            t = f2_sub(x[q][k], yk[k]);
            d2 = f2_fma(t, t, d2);
          }
          float a, b;
          f2_unpack(d2, a, b);
          if (LK == 0) {
            macc = fmaxf(macc, (FULL || v[2 * q]) ? a : 0.f);
            macc = fmaxf(macc, (FULL || v[2 * q + 1]) ? b : 0.f);
          } else {
            const float ra = (FULL || v[2 * q]) ? sqrt_approx(a) : 0.f;
            const float rb = (FULL || v[2 * q + 1]) ? sqrt_approx(b) : 0.f;
            part = f2_add(part, f2_pack(ra, rb));
          }
        }
      }
    }
    if (LK != 0) {
      part2 = f2_add(part2, part);
      if (++groups == 16) {
        float a, b;
        f2_unpack(part2, a, b);
        acc += (double)a + (double)b;
        part2 = 0ull;
        groups = 0;
      }
    }
  }
  if (LK != 0) {
    float a, b;
    f2_unpack(part2, a, b);
    acc += (double)a + (double)b;
  }
}

__device__ __forceinline__ float warp_maxf_big(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// per-dimension box of the valid points a warp holds (every lane gets it)
template <int D, int NP>
__device__ __forceinline__ void warp_box(const unsigned long long (&x)[NP][D],
                                         const bool (&v)[2 * NP], float (&lo)[D],
                                         float (&hi)[D]) {
#pragma unroll
  for (int k = 0; k < D; ++k) {
    lo[k] = INFINITY;
    hi[k] = -INFINITY;
#pragma unroll
    for (int h = 0; h < NP; ++h) {
      float a, b;
      f2_unpack(x[h][k], a, b);
      if (v[2 * h]) {
        lo[k] = fminf(lo[k], a);
        hi[k] = fmaxf(hi[k], a);
      }
      if (v[2 * h + 1]) {
        lo[k] = fminf(lo[k], b);
        hi[k] = fmaxf(hi[k], b);
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  }
}

// block-wide box of per-thread boxes into out[0, D) (lo) and out[D, 2D)
// (hi); the caller synchronises before reading it
template <int D>
__device__ __forceinline__ void block_box(float (&lo)[D], float (&hi)[D], float *out) {
  __shared__ float wb[BIG_TPB / 32][2 * D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      wb[w][k] = lo[k];
      wb[w][D + k] = hi[k];
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * D) {
    const int k = threadIdx.x;
    float m = wb[0][k];
    for (int i = 1; i < BIG_TPB / 32; ++i) m = k < D ? fminf(m, wb[i][k]) : fmaxf(m, wb[i][k]);
    out[k] = m;
  }
}

template <int LK, int D, int DP, int KIND>
__global__ void __launch_bounds__(BIG_TPB) k_big_eval32(State s, int r0) {
  constexpr int PPT = KIND == 0 ? (D <= 8 ? 8 : 4) : 2, NP = PPT / 2;
  __shared__ unsigned long long sh[BIG_TPB * D];
  __shared__ float boxs[2 * D];
  __shared__ double red[BIG_TPB / 32];
  __shared__ int sh_tile;
  const float *P = s.p32[s.cur];
  const int base = KIND == 0 ? 0 : s.bsched[BS_META + 1];  // kind 1 tiles follow kind 0's
  for (;;) {
    const int tile = bk_next(s, KIND, &sh_tile);
    if (tile < 0) break;
    int q0;
    const int r = r0 + bk_find(s, KIND, tile, q0);
    int sL = s.breq_sa[r], nL = s.breq_na[r], sS = s.breq_sb[r], nS = s.breq_nb[r];
    if (nS > nL) {
      int t0 = sL; sL = sS; sS = t0;
      t0 = nL; nL = nS; nS = t0;
    }
    const int sch = bk_chunk(KIND, nL, nS, D);
    const int ts = (nS + sch - 1) / sch;  // chunks of the smaller cluster
    const int sc0 = (q0 % ts) * sch, sc1 = min(nS, sc0 + sch);
    const int q = q0 / ts;
    unsigned long long x[NP][D];
    bool v[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) v[p] = q * (BIG_TPB * PPT) + p * BIG_TPB + (int)threadIdx.x < nL;
#pragma unroll
    for (int h = 0; h < NP; ++h) {
      const int l0 = q * (BIG_TPB * PPT) + (2 * h) * BIG_TPB + threadIdx.x;
      const int l1 = l0 + BIG_TPB;
#pragma unroll
      for (int k = 0; k < D; ++k)
        x[h][k] = f2_pack(v[2 * h] ? P[(size_t)(sL + l0) * DP + k] : 0.f,
                          v[2 * h + 1] ? P[(size_t)(sL + l1) * DP + k] : 0.f);
    }
    double acc = 0.0;
    float macc = 0.f;
    const bool full = v[PPT - 1];  // all points valid: no selects
    // complete linkage: the box of this warp's points, for skipping staged
    // chunks that cannot raise the pair's maximum
    float wlo[D], whi[D];
    int wpts = 0;  // valid points of this warp
    if (LK == 0) {
      warp_box<D, NP>(x, v, wlo, whi);
#pragma unroll
      for (int p = 0; p < PPT; ++p) wpts += v[p];
      wpts = __reduce_add_sync(0xffffffffu, wpts);
    }
    const int lq = r - r0;  // the request's slot in this batch
    for (int c0 = sc0; c0 < sc1; c0 += BIG_TPB) {
      const int cn = min(BIG_TPB, sc1 - c0);
      __syncthreads();
      float slo[D], shi[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        slo[k] = INFINITY;
        shi[k] = -INFINITY;
      }
      for (int i = threadIdx.x; i < cn * D; i += BIG_TPB) {
        const int j = i / D, k = i - j * D;
        const float y = P[(size_t)(sS + c0 + j) * DP + k];
        sh[i] = f2_pack(y, y);
        if (LK == 0) {
#pragma unroll
          for (int kk = 0; kk < D; ++kk)
            if (kk == k) {
              slo[kk] = fminf(slo[kk], y);
              shi[kk] = fmaxf(shi[kk], y);
            }
        }
      }
      if (LK == 0) block_box<D>(slo, shi, boxs);
      __syncthreads();
      if (LK == 0) {
        // every pair of this warp's points with the chunk is at most the
        // distance of the boxes' farthest corners; if that (rounded up and
        // widened by the FP32 error of a squared distance) is within a
        // maximum already computed for this pair, the chunk changes nothing
        float far2 = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float m = fmaxf(fmaxf(__fsub_ru(boxs[D + k], wlo[k]), __fsub_ru(whi[k], boxs[k])), 0.f);
          far2 = __fadd_ru(far2, __fmul_ru(m, m));
        }
        far2 = __fmul_ru(far2, 1.f + 2.f * (D + 4) * 5.9604645e-8f);
        const float seen = __shfl_sync(0xffffffffu, __int_as_float(*(volatile int *)&s.bmax2[lq]), 0);
        const float known = fmaxf(warp_maxf_big(macc), seen);
        if (far2 <= known) {  // uniform over the warp
          if ((threadIdx.x & 31) == 0)
            atomicAdd(&s.ctr->big_skip, (unsigned long long)wpts * (unsigned long long)cn);
          continue;
        }
      }
      if (full)
        big32_chunk<LK, D, NP, true>(sh, cn, x, v, acc, macc);
      else
        big32_chunk<LK, D, NP, false>(sh, cn, x, v, acc, macc);
    }
    if (LK == 0) {
      const float wm = warp_maxf_big(macc);
      if ((threadIdx.x & 31) == 0) atomicMax(&s.bmax2[lq], __float_as_int(wm));
    }
    bk_store<LK>(s, LK == 0 ? (double)macc : acc, red, base + tile);
  }
}

// CTAs that stay resident together: one wave (occupancy x SMs CTAs), tiles
// handed out dynamically; computed once per device and kernel (the cache is
// the caller's, one per instantiation)
struct GridCache {
  std::atomic<int> g[64];
};

template <typename F>
int resident_grid(F kernel, GridCache &c) {
  int dev = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  const bool cached = dev >= 0 && dev < 64;
  if (cached) {
    const int v = c.g[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, BIG_TPB, 0) != cudaSuccess) {
    cudaGetLastError();
    per = 1;
  }
  const int g = device_sms() * std::max(1, per);
  if (cached) c.g[dev].store(g, std::memory_order_relaxed);
  return g;
}

template <int LK, int D>
void launch_big32(const State &s, int r0, cudaStream_t st) {
  constexpr int DP = D <= 2 ? 2 : D <= 4 ? 4 : D <= 8 ? 8 : 16;
  static GridCache c0, c1;
  k_big_eval32<LK, D, DP, 0><<<resident_grid(k_big_eval32<LK, D, DP, 0>, c0), BIG_TPB, 0, st>>>(s, r0);
  k_big_eval32<LK, D, DP, 1><<<resident_grid(k_big_eval32<LK, D, DP, 1>, c1), BIG_TPB, 0, st>>>(s, r0);
}

template <int LK, int DP>
void launch_big64(const State &s, int r0, cudaStream_t st) {
  static GridCache c;
  k_big_eval64<LK, DP><<<resident_grid(k_big_eval64<LK, DP>, c), BIG_TPB, 0, st>>>(s, r0);
}

template <int LK>
int launch_big_lk(const State &s, int r0, cudaStream_t st) {
  switch (s.d) {  // FP32 requests, specialised on the true dimension
    case 1: launch_big32<LK, 1>(s, r0, st); break;
    case 2: launch_big32<LK, 2>(s, r0, st); break;
    case 3: launch_big32<LK, 3>(s, r0, st); break;
    case 4: launch_big32<LK, 4>(s, r0, st); break;
    case 5: launch_big32<LK, 5>(s, r0, st); break;
    case 6: launch_big32<LK, 6>(s, r0, st); break;
    case 7: launch_big32<LK, 7>(s, r0, st); break;
    case 8: launch_big32<LK, 8>(s, r0, st); break;
    case 9: launch_big32<LK, 9>(s, r0, st); break;
    case 10: launch_big32<LK, 10>(s, r0, st); break;
    case 11: launch_big32<LK, 11>(s, r0, st); break;
    case 12: launch_big32<LK, 12>(s, r0, st); break;
    case 13: launch_big32<LK, 13>(s, r0, st); break;
    case 14: launch_big32<LK, 14>(s, r0, st); break;
    case 15: launch_big32<LK, 15>(s, r0, st); break;
    case 16: launch_big32<LK, 16>(s, r0, st); break;
    default: return HAC_EINTERNAL;
  }
  switch (s.dp) {  // FP64 requests
    case 2: launch_big64<LK, 2>(s, r0, st); break;
    case 4: launch_big64<LK, 4>(s, r0, st); break;
    case 8: launch_big64<LK, 8>(s, r0, st); break;
    case 16: launch_big64<LK, 16>(s, r0, st); break;
    default: return HAC_EINTERNAL;
  }
  CK(cudaGetLastError());
  return HAC_OK;
}

}  // namespace
