// Longitude transforms of the SHT (Sec. B.3: "FFT along longitudes";
// Algorithm 1: 2 pi * FFT_1D_R2C followed by truncation to mmax).
//
// One CTA handles the mirror pair of latitude rows (k, nlat-1-k) for up to
// kFields fields.  The two real rows of a field are packed into one complex
// sequence z = u_k + i u_kbar, transformed by a mixed-radix (2, 3, 4, 5)
// Stockham FFT in shared memory, and separated with the conjugate symmetry
// of real transforms.  The analysis kernel writes the parity-folded
// coefficients E = F_k + F_kbar and O = F_k - F_kbar that the Legendre
// contraction consumes (Phat_l^m(-x) = (-1)^{l+m} Phat_l^m(x)); the
// synthesis kernel reads the folded G_even, G_odd back.
#include "sht_internal.cuh"

namespace shtgb {
namespace {

constexpr int kThreads = 256;
constexpr int kFields = 4;  // fields per CTA: 4 x 8 B = one 32 B sector per write

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }

// One Stockham pass with radix R over `nf` sequences of length n stored
// contiguously (sequence f at offset f * n).  Forward sign (e^{-2 pi i}).
// tw[q] = exp(-2 pi i q / n).
template <int R>
__device__ __forceinline__ void stockham_pass(const float2 *__restrict__ in, float2 *__restrict__ out,
                                              const float2 *__restrict__ tw, int n, int Ns, int nf) {
  const int nb = n / R;            // butterflies per sequence
  const int tstride = n / (Ns * R);  // twiddle index step
  for (int t = threadIdx.x; t < nb * nf; t += blockDim.x) {
    const int f = t / nb;
    const int j = t - f * nb;
    const float2 *src = in + f * n;
    float2 *dst = out + f * n;
    const int k = j % Ns;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; r++) v[r] = src[j + r * nb];
#pragma unroll
    for (int r = 1; r < R; r++) v[r] = cmul(v[r], tw[r * k * tstride]);
    float2 V[R];
    if (R == 2) {
      V[0] = cadd(v[0], v[1]);
      V[1] = csub(v[0], v[1]);
    } else if (R == 3) {
      const float h = 0.86602540378443864676f;  // sqrt(3) / 2
      float2 t1 = cadd(v[1], v[2]);
      float2 t2 = csub(v[0], cscale(t1, 0.5f));
      float2 t3 = cscale(csub(v[1], v[2]), h);  // multiplied by -i below
      V[0] = cadd(v[0], t1);
      V[1] = cadd(t2, mul_mi(t3));
      V[2] = csub(t2, mul_mi(t3));
    } else if (R == 4) {
      float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
      float2 b0 = cadd(v[1], v[3]), b1 = mul_mi(csub(v[1], v[3]));
      V[0] = cadd(a0, b0);
      V[1] = cadd(a1, b1);
      V[2] = csub(a0, b0);
      V[3] = csub(a1, b1);
    } else {  // R == 5
      const float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
      const float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
      const float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
      const float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
      float2 a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
      float2 a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
      V[0] = cadd(v[0], cadd(a1, a2));
      float2 r1 = make_float2(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
      float2 r2 = make_float2(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
      float2 q1 = make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y);
      float2 q2 = make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y);
      V[1] = cadd(r1, mul_mi(q1));
      V[4] = csub(r1, mul_mi(q1));
      V[2] = cadd(r2, mul_mi(q2));
      V[3] = csub(r2, mul_mi(q2));
    }
    const int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int q = 0; q < R; q++) dst[base + q * Ns] = V[q];
  }
}

// Forward FFT of nf sequences; returns the buffer that holds the result.
__device__ float2 *fft_forward(float2 *a, float2 *b, const float2 *tw, const RadixPlan &rp, int nf) {
  int Ns = 1;
  const int n = rp.n;
  for (int s = 0; s < rp.nstages; s++) {
    const int R = rp.r[s];
    if (R == 4) stockham_pass<4>(a, b, tw, n, Ns, nf);
    else if (R == 2) stockham_pass<2>(a, b, tw, n, Ns, nf);
    else if (R == 3) stockham_pass<3>(a, b, tw, n, Ns, nf);
    else stockham_pass<5>(a, b, tw, n, Ns, nf);
    __syncthreads();
    float2 *t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

__device__ __forceinline__ float mode_weight(int m, int n, int inverse_weights) {
  if (!inverse_weights) return 1.0f;
  if (m == 0) return 1.0f;
  if ((n & 1) == 0 && 2 * m == n) return 1.0f;
  return 2.0f;
}

// Output of the analysis: FP32 pairs, or bf16 hi/lo pairs (split).
struct OutF32 {
  float *F;
  __device__ __forceinline__ void put(int64_t idx, float2 v) const { *reinterpret_cast<float2 *>(F + idx) = v; }
};
struct OutBF16 {
  __nv_bfloat16 *hi, *lo;
  __device__ __forceinline__ void put(int64_t idx, float2 v) const {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
    *reinterpret_cast<__nv_bfloat162 *>(hi + idx) = h;
    if (lo) *reinterpret_cast<__nv_bfloat162 *>(lo + idx) = l;
  }
};

template <class Out>
__global__ void __launch_bounds__(kThreads)
r2c_pairs_kernel(const float *__restrict__ x, Out out, int nlat, int nlon, int M, int B, FoldLayout fl,
                 const float2 *__restrict__ twiddle, RadixPlan rp, const float *__restrict__ ring_scale,
                 int inverse_weights) {
  extern __shared__ float2 smem[];
  const int n = nlon;
  float2 *tw = smem;
  float2 *bufA = tw + n;
  float2 *bufB = bufA + kFields * n;
  const int kp = blockIdx.y;          // northern row k'
  const int ks = nlat - 1 - kp;       // mirrored southern row
  const bool equator = (kp == ks);
  const int b0 = blockIdx.x * kFields;
  const int nf = min(kFields, B - b0);

  for (int q = threadIdx.x; q < n; q += blockDim.x) tw[q] = twiddle[q];
  // pack rows: z = u_k + i u_kbar
  for (int f = 0; f < nf; f++) {
    const float *rn = x + ((int64_t)(b0 + f) * nlat + kp) * n;
    const float *rs = x + ((int64_t)(b0 + f) * nlat + ks) * n;
    float2 *z = bufA + f * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) z[j] = make_float2(rn[j], equator ? 0.f : rs[j]);
  }
  __syncthreads();
  float2 *Z = fft_forward(bufA, bufB, tw, rp, nf);

  const float sn = ring_scale ? ring_scale[kp] : 1.0f;
  const float ss = ring_scale ? ring_scale[ks] : 1.0f;
  // separate the two real transforms and fold by parity
  for (int t = threadIdx.x; t < nf * M; t += blockDim.x) {
    const int f = t / M;
    const int m = t - f * M;
    const float2 *zf = Z + f * n;
    const float2 zm = zf[m];
    const float2 zc = conjf2(zf[(n - m) % n]);
    const float c = 0.5f * mode_weight(m, n, inverse_weights);
    // X_k = (Z[m] + conj Z[n-m]) / 2 ; X_kbar = (Z[m] - conj Z[n-m]) / (2 i)
    float2 Fk = cscale(cadd(zm, zc), c * sn);
    float2 Fs = cscale(mul_mi(csub(zm, zc)), c * ss);
    float2 E, O;
    if (equator) {
      E = Fk;
      O = make_float2(0.f, 0.f);
    } else {
      E = cadd(Fk, Fs);
      O = csub(Fk, Fs);
    }
    const int64_t col = fold_col(fl, 2 * (int64_t)(b0 + f));
    out.put(fold_row(fl, m, 0, kp) + col, E);
    out.put(fold_row(fl, m, 1, kp) + col, O);
  }
}

__global__ void __launch_bounds__(kThreads)
c2r_pairs_kernel(const float *__restrict__ Gw, float *__restrict__ y, int nlat, int nlon, int M, int B, FoldLayout fl,
                 const float2 *__restrict__ twiddle, RadixPlan rp, const float *__restrict__ ring_scale,
                 int inverse_weights) {
  extern __shared__ float2 smem[];
  const int n = nlon;
  float2 *tw = smem;
  float2 *bufA = tw + n;
  float2 *bufB = bufA + kFields * n;
  const int kp = blockIdx.y;
  const int ks = nlat - 1 - kp;
  const bool equator = (kp == ks);
  const int b0 = blockIdx.x * kFields;
  const int nf = min(kFields, B - b0);
  const float sn = ring_scale ? ring_scale[kp] : 1.0f;
  const float ss = ring_scale ? ring_scale[ks] : 1.0f;

  for (int q = threadIdx.x; q < n; q += blockDim.x) tw[q] = twiddle[q];
  // Stage c_m / 2 * ring_scale * G for the northern row (bufA) and the
  // southern row (bufB) of each field; m < M <= n / 2 + 1 fits in n slots.
  for (int t = threadIdx.x; t < nf * M; t += blockDim.x) {
    const int f = t / M;
    const int m = t - f * M;
    const int64_t col = fold_col(fl, 2 * (int64_t)(b0 + f));
    const float2 ge = *reinterpret_cast<const float2 *>(Gw + fold_row(fl, m, 0, kp) + col);
    const float2 go = *reinterpret_cast<const float2 *>(Gw + fold_row(fl, m, 1, kp) + col);
    const float c = 0.5f * mode_weight(m, n, inverse_weights);
    float2 gn = equator ? ge : cadd(ge, go);
    float2 gs = equator ? make_float2(0.f, 0.f) : csub(ge, go);
    bufA[f * n + m] = cscale(gn, c * sn);
    bufB[f * n + m] = cscale(gs, c * ss);
  }
  __syncthreads();
  // Hermitian extension of each row, H(q) = G(q) [q < M] + conj G(n - q)
  // [(n - q) mod n < M], so that u_j = sum_q H(q) e^{2 pi i j q / n} is real.
  // Both rows are packed as Z = H_north + i H_south, and the inverse DFT is
  // evaluated as conj(FFT(conj Z)).  conj Z goes to the third buffer Zc.
  float2 *Zc = bufB + kFields * n;
  for (int t = threadIdx.x; t < nf * n; t += blockDim.x) {
    const int f = t / n;
    const int q = t - f * n;
    float2 hn = make_float2(0.f, 0.f), hs = make_float2(0.f, 0.f);
    if (q < M) {
      hn = cadd(hn, bufA[f * n + q]);
      hs = cadd(hs, bufB[f * n + q]);
    }
    const int qm = (n - q) % n;
    if (qm < M) {
      hn = cadd(hn, conjf2(bufA[f * n + qm]));
      hs = cadd(hs, conjf2(bufB[f * n + qm]));
    }
    // Z = hn + i hs
    const float2 z = make_float2(hn.x - hs.y, hn.y + hs.x);
    Zc[f * n + q] = conjf2(z);
  }
  __syncthreads();
  float2 *out = fft_forward(Zc, bufA, tw, rp, nf);
  // z = conj(out): real part -> northern row, imaginary part -> southern row
  for (int f = 0; f < nf; f++) {
    float *rn = y + ((int64_t)(b0 + f) * nlat + kp) * n;
    float *rs = y + ((int64_t)(b0 + f) * nlat + ks) * n;
    const float2 *of = out + f * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const float2 v = of[j];
      rn[j] = v.x;
      if (!equator) rs[j] = -v.y;
    }
  }
}

// Longitude analysis of arbitrary latitude rows (the local step of the
// distributed transform, where a rank holds a block of latitudes and no
// mirror pairs): rows r = 0 .. R-1 of x[R][nlon], row r on latitude
// k0 + (r mod nrows) of the grid; rows 2q and 2q + 1 share one complex
// sequence z = u_2q + i u_2q+1, separated after the FFT.  F[r][m], m < M,
// times ring_scale of the row's latitude; no parity fold.
__global__ void __launch_bounds__(kThreads)
r2c_rows_kernel(const float *__restrict__ x, float2 *__restrict__ F, int64_t R, int nrows, int k0, int nlon, int M,
                const float2 *__restrict__ twiddle, RadixPlan rp, const float *__restrict__ ring_scale) {
  extern __shared__ float2 smem[];
  const int n = nlon;
  float2 *tw = smem;
  float2 *bufA = tw + n;
  float2 *bufB = bufA + kFields * n;
  const int64_t r0 = (int64_t)blockIdx.x * 2 * kFields;
  const int64_t pending = (R - r0 + 1) / 2;
  const int nf = pending < kFields ? (int)pending : kFields;
  for (int q = threadIdx.x; q < n; q += blockDim.x) tw[q] = twiddle[q];
  for (int f = 0; f < nf; f++) {
    const int64_t ra = r0 + 2 * f, rb = ra + 1;
    const float *xa = x + ra * n;
    const float *xb = x + rb * n;
    float2 *z = bufA + f * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) z[j] = make_float2(xa[j], rb < R ? xb[j] : 0.f);
  }
  __syncthreads();
  float2 *Z = fft_forward(bufA, bufB, tw, rp, nf);
  for (int t = threadIdx.x; t < nf * M; t += blockDim.x) {
    const int f = t / M;
    const int m = t - f * M;
    const int64_t ra = r0 + 2 * f, rb = ra + 1;
    const float2 *zf = Z + f * n;
    const float2 zm = zf[m];
    const float2 zc = conjf2(zf[(n - m) % n]);
    const float sa = ring_scale[k0 + (int)(ra % nrows)];
    F[ra * M + m] = cscale(cadd(zm, zc), 0.5f * sa);
    if (rb < R) {
      const float sb = ring_scale[k0 + (int)(rb % nrows)];
      F[rb * M + m] = cscale(mul_mi(csub(zm, zc)), 0.5f * sb);
    }
  }
}

// Longitude synthesis of arbitrary rows: y[r][j] = sum_{m < M} c_m Re(G[r][m]
// e^{2 pi i j m / nlon}) (c_0 = 1, c_{nlon/2} = 1, c_m = 2 otherwise; the
// imaginary parts of m = 0 and of the Nyquist mode are ignored), two rows
// per complex sequence.
__global__ void __launch_bounds__(kThreads)
c2r_rows_kernel(const float2 *__restrict__ G, float *__restrict__ y, int64_t R, int nlon, int M,
                const float2 *__restrict__ twiddle, RadixPlan rp) {
  extern __shared__ float2 smem[];
  const int n = nlon;
  float2 *tw = smem;
  float2 *bufA = tw + n;
  float2 *bufB = bufA + kFields * n;
  float2 *Zc = bufB + kFields * n;
  const int64_t r0 = (int64_t)blockIdx.x * 2 * kFields;
  const int64_t pending = (R - r0 + 1) / 2;
  const int nf = pending < kFields ? (int)pending : kFields;
  for (int q = threadIdx.x; q < n; q += blockDim.x) tw[q] = twiddle[q];
  for (int t = threadIdx.x; t < nf * M; t += blockDim.x) {
    const int f = t / M;
    const int m = t - f * M;
    const int64_t ra = r0 + 2 * f, rb = ra + 1;
    const float c = 0.5f * mode_weight(m, n, 1);
    bufA[f * n + m] = cscale(G[ra * M + m], c);
    bufB[f * n + m] = rb < R ? cscale(G[rb * M + m], c) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nf * n; t += blockDim.x) {
    const int f = t / n;
    const int q = t - f * n;
    float2 ha = make_float2(0.f, 0.f), hb = make_float2(0.f, 0.f);
    if (q < M) {
      ha = cadd(ha, bufA[f * n + q]);
      hb = cadd(hb, bufB[f * n + q]);
    }
    const int qm = (n - q) % n;
    if (qm < M) {
      ha = cadd(ha, conjf2(bufA[f * n + qm]));
      hb = cadd(hb, conjf2(bufB[f * n + qm]));
    }
    const float2 z = make_float2(ha.x - hb.y, ha.y + hb.x);  // Z = ha + i hb
    Zc[f * n + q] = conjf2(z);
  }
  __syncthreads();
  float2 *out = fft_forward(Zc, bufA, tw, rp, nf);
  for (int f = 0; f < nf; f++) {
    const int64_t ra = r0 + 2 * f, rb = ra + 1;
    const float2 *of = out + f * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const float2 v = of[j];
      y[ra * n + j] = v.x;
      if (rb < R) y[rb * n + j] = -v.y;
    }
  }
}

}  // namespace

static size_t fft_smem_bytes(int nlon, int nbuf) {
  return sizeof(float2) * (size_t)nlon * (1 + (size_t)nbuf * kFields);
}

static cudaError_t set_smem(const void *fn, size_t bytes) {
  if (bytes > 48 * 1024)
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

cudaError_t launch_r2c(const float *x, float *Fw, int nlat, int nlon, int M, int B, FoldLayout fl,
                       const float2 *twiddle, const RadixPlan &rp, const float *ring_scale, int inverse_weights,
                       cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  const int Kh = (nlat + 1) / 2;
  dim3 grid((B + kFields - 1) / kFields, Kh);
  size_t smem = fft_smem_bytes(nlon, 2);
  cudaError_t e = set_smem((const void *)r2c_pairs_kernel<OutF32>, smem);
  if (e != cudaSuccess) return e;
  r2c_pairs_kernel<OutF32><<<grid, kThreads, smem, st>>>(x, OutF32{Fw}, nlat, nlon, M, B, fl, twiddle, rp,
                                                         ring_scale, inverse_weights);
  return cudaGetLastError();
}

cudaError_t launch_r2c_bf16(const float *x, __nv_bfloat16 *Fhi, __nv_bfloat16 *Flo, int nlat, int nlon, int M, int B,
                            FoldLayout fl, const float2 *twiddle, const RadixPlan &rp, const float *ring_scale,
                            int inverse_weights, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  const int Kh = (nlat + 1) / 2;
  dim3 grid((B + kFields - 1) / kFields, Kh);
  size_t smem = fft_smem_bytes(nlon, 2);
  cudaError_t e = set_smem((const void *)r2c_pairs_kernel<OutBF16>, smem);
  if (e != cudaSuccess) return e;
  r2c_pairs_kernel<OutBF16><<<grid, kThreads, smem, st>>>(x, OutBF16{Fhi, Flo}, nlat, nlon, M, B, fl, twiddle, rp,
                                                          ring_scale, inverse_weights);
  return cudaGetLastError();
}

cudaError_t launch_c2r(const float *Gw, float *y, int nlat, int nlon, int M, int B, FoldLayout fl,
                       const float2 *twiddle, const RadixPlan &rp, const float *ring_scale, int inverse_weights,
                       cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  const int Kh = (nlat + 1) / 2;
  dim3 grid((B + kFields - 1) / kFields, Kh);
  size_t smem = fft_smem_bytes(nlon, 3);
  cudaError_t e = set_smem((const void *)c2r_pairs_kernel, smem);
  if (e != cudaSuccess) return e;
  c2r_pairs_kernel<<<grid, kThreads, smem, st>>>(Gw, y, nlat, nlon, M, B, fl, twiddle, rp, ring_scale,
                                                 inverse_weights);
  return cudaGetLastError();
}

cudaError_t launch_r2c_rows(const float *x, float2 *F, int64_t R, int nrows, int k0, int nlon, int M,
                            const float2 *twiddle, const RadixPlan &rp, const float *ring_scale, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  const int64_t nblk = (R + 2 * kFields - 1) / (2 * kFields);
  if (nblk > 0x7fffffff) return cudaErrorInvalidValue;
  const size_t smem = fft_smem_bytes(nlon, 2);
  cudaError_t e = set_smem((const void *)r2c_rows_kernel, smem);
  if (e != cudaSuccess) return e;
  r2c_rows_kernel<<<(unsigned)nblk, kThreads, smem, st>>>(x, F, R, nrows, k0, nlon, M, twiddle, rp, ring_scale);
  return cudaGetLastError();
}

cudaError_t launch_c2r_rows(const float2 *G, float *y, int64_t R, int nlon, int M, const float2 *twiddle,
                            const RadixPlan &rp, cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  const int64_t nblk = (R + 2 * kFields - 1) / (2 * kFields);
  if (nblk > 0x7fffffff) return cudaErrorInvalidValue;
  const size_t smem = fft_smem_bytes(nlon, 3);
  cudaError_t e = set_smem((const void *)c2r_rows_kernel, smem);
  if (e != cudaSuccess) return e;
  c2r_rows_kernel<<<(unsigned)nblk, kThreads, smem, st>>>(G, y, R, nlon, M, twiddle, rp);
  return cudaGetLastError();
}

}  // namespace shtgb
