// Longitude transforms for nlon = 45 P (P = 4, 8, 16, 32: the 2, 1, 0.5 and
// 0.25 degree grids with nlon = 180, 360, 720, 1440), as a "four-step" FFT
// with the whole sequence in registers:
//   n = t + P j (lane t < P, register j < 45),  k = k2 + 45 k1,
//   X[k2 + 45 k1] = sum_t w_P^{t k1} w_N^{t k2} sum_j x[t + P j] w_45^{j k2}.
// Each lane does one 45-point DFT in registers (radices 5, 3, 3), multiplies
// by w_N^{t k2}, writes the 45 values to a padded row-per-k2 buffer, and then
// runs P-point DFTs (radix 4/2, in registers) on the rows it owns, writing
// them back in place.  Only warp-level synchronisation is needed inside a
// transform.  As in the generic kernels, the two mirror rows (k, nlat-1-k) of
// one field are packed into one complex sequence and separated afterwards;
// a CTA handles 8 fields of 32 / P ring pairs so that the folded output rows
// are written in contiguous 8-field segments.
#include <algorithm>

#include "sht_internal.cuh"
#include "tc_common.cuh"

namespace shtgb {
namespace {

constexpr int kQ = 45;
constexpr int kThreads = 256;
constexpr int kFB = 8;  // fields per CTA

// exp(-2 pi i k / 45), k = 0..44 (rounded from double precision)
__constant__ float2 kRoot45[45] = {
    {1.000000000e+00f, 0.000000000e+00f}, {9.902680687e-01f, -1.391731010e-01f}, {9.612616959e-01f, -2.756373558e-01f},
    {9.135454576e-01f, -4.067366431e-01f}, {8.480480962e-01f, -5.299192642e-01f}, {7.660444431e-01f, -6.427876097e-01f},
    {6.691306064e-01f, -7.431448255e-01f}, {5.591929035e-01f, -8.290375726e-01f}, {4.383711468e-01f, -8.987940463e-01f},
    {3.090169944e-01f, -9.510565163e-01f}, {1.736481777e-01f, -9.848077530e-01f}, {3.489949670e-02f, -9.993908270e-01f},
    {-1.045284633e-01f, -9.945218954e-01f}, {-2.419218956e-01f, -9.702957263e-01f}, {-3.746065934e-01f, -9.271838546e-01f},
    {-5.000000000e-01f, -8.660254038e-01f}, {-6.156614753e-01f, -7.880107536e-01f}, {-7.193398003e-01f, -6.946583705e-01f},
    {-8.090169944e-01f, -5.877852523e-01f}, {-8.829475929e-01f, -4.694715628e-01f}, {-9.396926208e-01f, -3.420201433e-01f},
    {-9.781476007e-01f, -2.079116908e-01f}, {-9.975640503e-01f, -6.975647374e-02f}, {-9.975640503e-01f, 6.975647374e-02f},
    {-9.781476007e-01f, 2.079116908e-01f}, {-9.396926208e-01f, 3.420201433e-01f}, {-8.829475929e-01f, 4.694715628e-01f},
    {-8.090169944e-01f, 5.877852523e-01f}, {-7.193398003e-01f, 6.946583705e-01f}, {-6.156614753e-01f, 7.880107536e-01f},
    {-5.000000000e-01f, 8.660254038e-01f}, {-3.746065934e-01f, 9.271838546e-01f}, {-2.419218956e-01f, 9.702957263e-01f},
    {-1.045284633e-01f, 9.945218954e-01f}, {3.489949670e-02f, 9.993908270e-01f}, {1.736481777e-01f, 9.848077530e-01f},
    {3.090169944e-01f, 9.510565163e-01f}, {4.383711468e-01f, 8.987940463e-01f}, {5.591929035e-01f, 8.290375726e-01f},
    {6.691306064e-01f, 7.431448255e-01f}, {7.660444431e-01f, 6.427876097e-01f}, {8.480480962e-01f, 5.299192642e-01f},
    {9.135454576e-01f, 4.067366431e-01f}, {9.612616959e-01f, 2.756373558e-01f}, {9.902680687e-01f, 1.391731010e-01f},
};
// exp(-2 pi i k / 32), k = 0..31 (rounded from double precision)
__constant__ float2 kRoot32[32] = {
    {1.000000000e+00f, 0.000000000e+00f}, {9.807852804e-01f, -1.950903220e-01f}, {9.238795325e-01f, -3.826834324e-01f},
    {8.314696123e-01f, -5.555702330e-01f}, {7.071067812e-01f, -7.071067812e-01f}, {5.555702330e-01f, -8.314696123e-01f},
    {3.826834324e-01f, -9.238795325e-01f}, {1.950903220e-01f, -9.807852804e-01f}, {0.000000000e+00f, -1.000000000e+00f},
    {-1.950903220e-01f, -9.807852804e-01f}, {-3.826834324e-01f, -9.238795325e-01f}, {-5.555702330e-01f, -8.314696123e-01f},
    {-7.071067812e-01f, -7.071067812e-01f}, {-8.314696123e-01f, -5.555702330e-01f}, {-9.238795325e-01f, -3.826834324e-01f},
    {-9.807852804e-01f, -1.950903220e-01f}, {-1.000000000e+00f, 0.000000000e+00f}, {-9.807852804e-01f, 1.950903220e-01f},
    {-9.238795325e-01f, 3.826834324e-01f}, {-8.314696123e-01f, 5.555702330e-01f}, {-7.071067812e-01f, 7.071067812e-01f},
    {-5.555702330e-01f, 8.314696123e-01f}, {-3.826834324e-01f, 9.238795325e-01f}, {-1.950903220e-01f, 9.807852804e-01f},
    {0.000000000e+00f, 1.000000000e+00f}, {1.950903220e-01f, 9.807852804e-01f}, {3.826834324e-01f, 9.238795325e-01f},
    {5.555702330e-01f, 8.314696123e-01f}, {7.071067812e-01f, 7.071067812e-01f}, {8.314696123e-01f, 5.555702330e-01f},
    {9.238795325e-01f, 3.826834324e-01f}, {9.807852804e-01f, 1.950903220e-01f},
};

// Complex additions and real scalings on the packed two-lane FP32
// instructions (one instruction for the real and imaginary parts; each lane
// rounds as the scalar operation does; a - b as b (-1) + a, exact up to the
// one rounding).  The complex product stays scalar: its packed forms need
// operand swaps that cost as much as they save (timed on the 45 P grids).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
// a + s b
__device__ __forceinline__ float2 caxpy(float s, float2 b, float2 a) { return __ffma2_rn(make_float2(s, s), b, a); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }

template <int N>
__device__ __forceinline__ float2 root(int k);
template <>
__device__ __forceinline__ float2 root<9>(int k) { return kRoot45[(5 * k) % 45]; }
template <>
__device__ __forceinline__ float2 root<32>(int k) { return kRoot32[k & 31]; }
template <>
__device__ __forceinline__ float2 root<16>(int k) { return kRoot32[(k & 15) * 2]; }
template <>
__device__ __forceinline__ float2 root<8>(int k) { return kRoot32[(k & 7) * 4]; }
template <>
__device__ __forceinline__ float2 root<4>(int k) { return kRoot32[(k & 3) * 8]; }

// forward R-point DFT in place
template <int R>
__device__ __forceinline__ void butterfly(float2 (&v)[R]) {
  if (R == 2) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if (R == 3) {
    const float h = 0.86602540378443864676f;
    const float2 t1 = cadd(v[1], v[2]);
    const float2 t2 = caxpy(-0.5f, t1, v[0]);
    const float2 t3 = mul_mi(cscale(csub(v[1], v[2]), h));
    v[0] = cadd(v[0], t1);
    v[1] = cadd(t2, t3);
    v[2] = csub(t2, t3);
  } else if (R == 4) {
    const float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    const float2 b0 = cadd(v[1], v[3]), b1 = mul_mi(csub(v[1], v[3]));
    v[0] = cadd(a0, b0);
    v[1] = cadd(a1, b1);
    v[2] = csub(a0, b0);
    v[3] = csub(a1, b1);
  } else if (R == 5) {
    const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
    const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
    const float2 a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
    const float2 a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    const float2 r1 = caxpy(c2, a2, caxpy(c1, a1, v[0]));
    const float2 r2 = caxpy(c1, a2, caxpy(c2, a1, v[0]));
    const float2 q1 = mul_mi(caxpy(s2, b2, cscale(b1, s1)));
    const float2 q2 = mul_mi(caxpy(-s1, b2, cscale(b1, s2)));
    v[0] = cadd(v[0], cadd(a1, a2));
    v[1] = cadd(r1, q1);
    v[4] = csub(r1, q1);
    v[2] = cadd(r2, q2);
    v[3] = csub(r2, q2);
  }
}

// One Stockham stage (radix R, current span Ns) of an N-point DFT held in
// registers; all indices are compile-time after unrolling.
template <int N, int Ns, int R>
__device__ __forceinline__ void reg_stage(float2 (&a)[N]) {
  float2 t[N];
#pragma unroll
  for (int j = 0; j < N / R; j++) {
    const int k = j % Ns;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
      v[r] = a[j + r * (N / R)];
      if (r > 0 && k > 0) v[r] = cmul(v[r], root<N>(r * k * (N / (Ns * R))));
    }
    butterfly<R>(v);
    const int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int q = 0; q < R; q++) t[base + q * Ns] = v[q];
  }
#pragma unroll
  for (int i = 0; i < N; i++) a[i] = t[i];
}

template <int N>
struct RegDFT;
template <>
struct RegDFT<9> {
  static __device__ __forceinline__ void run(float2 (&a)[9]) {
    reg_stage<9, 1, 3>(a);
    reg_stage<9, 3, 3>(a);
  }
};
// 45 = 9 x 5 with coprime factors (Good-Thomas): inputs n = (5 n1 + 9 n2)
// mod 45, outputs k = (10 k1 + 36 k2) mod 45 (k = k1 mod 9, k = k2 mod 5),
// 9-point DFTs along n1 and 5-point DFTs along n2, no twiddles between them.
template <>
struct RegDFT<45> {
  static __device__ __forceinline__ void run(float2 (&a)[45]) {
    float2 b[9][5];
#pragma unroll
    for (int n2 = 0; n2 < 5; n2++) {
      float2 c[9];
#pragma unroll
      for (int n1 = 0; n1 < 9; n1++) c[n1] = a[(5 * n1 + 9 * n2) % 45];
      RegDFT<9>::run(c);
#pragma unroll
      for (int k1 = 0; k1 < 9; k1++) b[k1][n2] = c[k1];
    }
#pragma unroll
    for (int k1 = 0; k1 < 9; k1++) {
      float2 c[5];
#pragma unroll
      for (int n2 = 0; n2 < 5; n2++) c[n2] = b[k1][n2];
      butterfly<5>(c);
#pragma unroll
      for (int k2 = 0; k2 < 5; k2++) a[(10 * k1 + 36 * k2) % 45] = c[k2];
    }
  }
};
template <>
struct RegDFT<32> {
  static __device__ __forceinline__ void run(float2 (&a)[32]) {
    reg_stage<32, 1, 4>(a);
    reg_stage<32, 4, 4>(a);
    reg_stage<32, 16, 2>(a);
  }
};
template <>
struct RegDFT<16> {
  static __device__ __forceinline__ void run(float2 (&a)[16]) {
    reg_stage<16, 1, 4>(a);
    reg_stage<16, 4, 4>(a);
  }
};
template <>
struct RegDFT<8> {
  static __device__ __forceinline__ void run(float2 (&a)[8]) {
    reg_stage<8, 1, 4>(a);
    reg_stage<8, 4, 2>(a);
  }
};
template <>
struct RegDFT<4> {
  static __device__ __forceinline__ void run(float2 (&a)[4]) { reg_stage<4, 1, 4>(a); }
};

// Buffer of one sequence: rows k2 < 45 of rpitch entries, P + 1 (padding
// against bank conflicts) except for P = 4, whose 4 lanes per sequence meet
// distinct banks unpadded and whose 64 sequences per CTA must fit twice per
// SM.  After seq_fft, X[k2 + 45 k1] sits at row k2, column k1.
template <int P>
__host__ __device__ constexpr int rpitch() {
  return P == 4 ? P : P + 1;
}
// Sequence buffer pitch (float2 entries): 45 rows, padded to 2 mod 16 so
// that the 8 fields of a CTA fall on distinct bank pairs.
template <int P>
__host__ __device__ constexpr int seq_pitch() {
  return (kQ * rpitch<P>() + 15 - 2) / 16 * 16 + 2;
}

// Twiddle table w_N^{t k2} (t < P, k2 < 45, lane-major) into shared memory
// from the plan's table w_N^q; indices walked without divisions.
template <int P>
__device__ __forceinline__ void load_twiddles(float2 *tw, const float2 *__restrict__ twiddle) {
  constexpr int N = kQ * P;
  int d = threadIdx.x / kQ, r = threadIdx.x - (threadIdx.x / kQ) * kQ;  // q = 45 d + r
  constexpr int kStepD = kThreads / kQ, kStepR = kThreads % kQ;
  for (int q = threadIdx.x; q < N; q += kThreads) {
    tw[q] = twiddle[d * r];
    r += kStepR;
    d += kStepD;
    if (r >= kQ) {
      r -= kQ;
      d++;
    }
  }
}

template <int P>
__device__ __forceinline__ int spec_index(int k) {
  return (k % kQ) * rpitch<P>() + k / kQ;
}

// Forward DFT of the sequence held as v[j] = z[t + P j] by lane t.
// twT[t * 45 + k2] = w_N^{t k2} (lane-major, so that the lanes of one k2 hit
// distinct banks).
template <int P>
__device__ __forceinline__ void seq_fft(float2 (&v)[kQ], int t, float2 *buf, const float2 *twT) {
  RegDFT<kQ>::run(v);
#pragma unroll
  for (int k2 = 1; k2 < kQ; k2++) v[k2] = cmul(v[k2], twT[t * kQ + k2]);
#pragma unroll
  for (int k2 = 0; k2 < kQ; k2++) buf[k2 * rpitch<P>() + t] = v[k2];
  __syncwarp();
  for (int k2 = t; k2 < kQ; k2 += P) {
    float2 u[P];
#pragma unroll
    for (int n = 0; n < P; n++) u[n] = buf[k2 * rpitch<P>() + n];
    RegDFT<P>::run(u);
#pragma unroll
    for (int n = 0; n < P; n++) buf[k2 * rpitch<P>() + n] = u[n];
  }
  __syncwarp();
}

// Destinations of the analysis: `put` writes one complex value, `put2` the
// values of two adjacent fields (idx a multiple of 4 elements).
struct OutF32 {
  float *F;
  __device__ __forceinline__ void put(int64_t idx, float2 v) const { *reinterpret_cast<float2 *>(F + idx) = v; }
  __device__ __forceinline__ void put2(int64_t idx, float2 a, float2 b) const {
    *reinterpret_cast<float4 *>(F + idx) = make_float4(a.x, a.y, b.x, b.y);
  }
};
struct OutBF16 {
  __nv_bfloat16 *hi, *lo;
  __device__ __forceinline__ void put(int64_t idx, float2 v) const {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
    *reinterpret_cast<__nv_bfloat162 *>(hi + idx) = h;
    if (lo) {
      const float2 hf = __bfloat1622float2(h);
      *reinterpret_cast<__nv_bfloat162 *>(lo + idx) = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
    }
  }
  __device__ __forceinline__ void put2(int64_t idx, float2 a, float2 b) const {
    const __nv_bfloat162 ha = __floats2bfloat162_rn(a.x, a.y), hb = __floats2bfloat162_rn(b.x, b.y);
    *reinterpret_cast<uint2 *>(hi + idx) =
        make_uint2(*reinterpret_cast<const uint32_t *>(&ha), *reinterpret_cast<const uint32_t *>(&hb));
    if (lo) {
      const float2 da = csub(a, __bfloat1622float2(ha)), db = csub(b, __bfloat1622float2(hb));
      const __nv_bfloat162 la = __floats2bfloat162_rn(da.x, da.y);
      const __nv_bfloat162 lb = __floats2bfloat162_rn(db.x, db.y);
      *reinterpret_cast<uint2 *>(lo + idx) =
          make_uint2(*reinterpret_cast<const uint32_t *>(&la), *reinterpret_cast<const uint32_t *>(&lb));
    }
  }
};

// Output stage of the analysis: separate the two real transforms of every
// sequence buffer in `bufs`, fold by parity, write 8-field segments: thread
// (f2, m0) handles fields 2 f2, 2 f2 + 1 and orders m0, m0 + 64, ... (m =
// 45 q + r tracked without divisions).
template <int P, class Out>
__device__ __forceinline__ void r2c45_emit(int bx, int by, const float2 *bufs, Out out, int nlat, int M, int B,
                                           FoldLayout fl, const float *__restrict__ ring_scale, int inverse_weights,
                                           int tid) {
  constexpr int N = kQ * P;
  constexpr int NPAIR = kThreads / P / kFB;
  constexpr int BUF = seq_pitch<P>();
  constexpr int kPairs = kFB / 2;
  constexpr int kMStep = kThreads / kPairs;  // 64
  const int Kh = (nlat + 1) / 2;
  const int b0 = bx * kFB;
  const int f2 = tid % kPairs, m0 = tid / kPairs;
  const int fa = 2 * f2;
  if (b0 + fa >= B) return;
  const bool two = b0 + fa + 1 < B;
  const int64_t col = fold_col(fl, 2 * (int64_t)(b0 + fa));  // 4 columns of one 16-column group
  const int64_t pstride = fl.sp;                            // E row -> O row
#pragma unroll 1
  for (int pq = 0; pq < NPAIR; pq++) {
    const int kq = by * NPAIR + pq;
    if (kq >= Kh) continue;
    const int kqs = nlat - 1 - kq;
    const bool eqr = kq == kqs;
    const float sn = 0.5f * (ring_scale ? ring_scale[kq] : 1.0f);
    const float ss = 0.5f * (ring_scale ? ring_scale[kqs] : 1.0f);
    const float2 *Za = bufs + (pq * kFB + fa) * BUF;
    const float2 *Zb = Za + BUF;
    int r = m0 % kQ, q = m0 / kQ;
    int64_t o = fold_row(fl, m0, 0, kq) + col;
#pragma unroll 2
    for (int m = m0; m < M; m += kMStep, o += kMStep * fl.sm) {
      // X[m] sits at spec_index(m); X[N - m] at spec_index(N - m)
      const int im = r * rpitch<P>() + q;
      const int ic = m == 0 ? 0 : (r > 0 ? (kQ - r) * rpitch<P>() + (P - 1 - q) : P - q);
      const float w = (inverse_weights && m != 0 && 2 * m != N) ? 2.0f : 1.0f;
      const float wn = w * sn, ws = w * ss;
      float2 e[2], od[2];
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const float2 *Z = h ? Zb : Za;
        const float2 zm = Z[im];
        const float2 zc = conjf2(Z[ic]);
        const float2 Fk = cscale(cadd(zm, zc), wn);
        const float2 Fs = cscale(mul_mi(csub(zm, zc)), ws);
        e[h] = eqr ? Fk : cadd(Fk, Fs);
        od[h] = eqr ? make_float2(0.f, 0.f) : csub(Fk, Fs);
      }
      if (two) {
        out.put2(o, e[0], e[1]);
        out.put2(o + pstride, od[0], od[1]);
      } else {
        out.put(o, e[0]);
        out.put(o + pstride, od[0]);
      }
      // m += 64 = 45 + 19
      r += kMStep - kQ;
      q++;
      if (r >= kQ) {
        r -= kQ;
        q++;
      }
    }
  }
}

// One CTA of the analysis: fields bx kFB .. bx kFB + 7, ring pairs
// by NPAIR .. by NPAIR + NPAIR - 1.
template <int P, class Out>
__device__ __forceinline__ void r2c45_body(int bx, int by, const float *__restrict__ x, Out out, int nlat, int M,
                                           int B, FoldLayout fl, const float2 *__restrict__ twiddle,
                                           const float *__restrict__ ring_scale, int inverse_weights) {
  constexpr int N = kQ * P;
  constexpr int NPAIR = kThreads / P / kFB;
  constexpr int BUF = seq_pitch<P>();
  extern __shared__ float2 smem[];
  float2 *tw = smem;
  float2 *bufs = smem + N;
  const int Kh = (nlat + 1) / 2;
  const int s = threadIdx.x / P, t = threadIdx.x % P;
  const int f = s % kFB, pp = s / kFB;
  const int b = bx * kFB + f;
  const int kp = by * NPAIR + pp;
  const int ks = nlat - 1 - kp;
  const bool live = (b < B) && (kp < Kh);
  load_twiddles<P>(tw, twiddle);
  float2 v[kQ];
  if (live) {
    const float *rn = x + ((int64_t)b * nlat + kp) * N;
    const float *rs = x + ((int64_t)b * nlat + ks) * N;
    const bool eq = (kp == ks);
#pragma unroll
    for (int j = 0; j < kQ; j++) v[j] = make_float2(__ldg(rn + t + P * j), eq ? 0.f : __ldg(rs + t + P * j));
  } else {
#pragma unroll
    for (int j = 0; j < kQ; j++) v[j] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  float2 *buf = bufs + s * BUF;
  seq_fft<P>(v, t, buf, tw);
  __syncthreads();
  r2c45_emit<P, Out>(bx, by, bufs, out, nlat, M, B, fl, ring_scale, inverse_weights, threadIdx.x);
}

template <int P, class Out>
__global__ void __launch_bounds__(kThreads, 2)
r2c45_kernel(const float *__restrict__ x, Out out, int nlat, int M, int B, FoldLayout fl, const float2 *__restrict__ twiddle,
             const float *__restrict__ ring_scale, int inverse_weights) {
  r2c45_body<P, Out>(blockIdx.x, blockIdx.y, x, out, nlat, M, B, fl, twiddle, ring_scale, inverse_weights);
}

// Synthesis staging of one item: conj(Z) (c_m / 2 * ring scale * G of the
// northern and southern rows, as the Hermitian sequences' Z = H_n + i H_s)
// of fields fa, fa + 1 at order m of ring pair kq, from their E and O
// values ge, go (two fields' complex values each), into the two sequence
// buffers at Ba.
template <int P>
__device__ __forceinline__ void c2r45_put(float2 *Ba, float4 ge, float4 go, int m, int kq, int nlat,
                                          const float *__restrict__ ring_scale, int inverse_weights) {
  constexpr int N = kQ * P;
  constexpr int BUF = seq_pitch<P>();
  const int kqs = nlat - 1 - kq;
  const bool eq = (kq == kqs);
  const float sn = 0.5f * (ring_scale ? ring_scale[kq] : 1.0f);
  const float ss = 0.5f * (ring_scale ? ring_scale[kqs] : 1.0f);
  const float w = (inverse_weights && m != 0 && 2 * m != N) ? 2.0f : 1.0f;
  const int mq = m == 0 ? 0 : N - m;
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const float2 e = h ? make_float2(ge.z, ge.w) : make_float2(ge.x, ge.y);
    const float2 o = h ? make_float2(go.z, go.w) : make_float2(go.x, go.y);
    const float2 gn = cscale(eq ? e : cadd(e, o), w * sn);
    const float2 gs = eq ? make_float2(0.f, 0.f) : cscale(csub(e, o), w * ss);
    // Z = H_n + i H_s of the Hermitian extensions, stored conjugated:
    // G_m enters Z[m], conj(G_m) enters Z[N - m]
    const float2 za = make_float2(gn.x - gs.y, -(gn.y + gs.x));
    const float2 zb = make_float2(gn.x + gs.y, gn.y - gs.x);
    float2 *Bq = Ba + h * BUF;
    if (mq == m) {
      Bq[m] = cadd(za, zb);
    } else {
      Bq[m] = za;
      Bq[mq] = zb;
    }
  }
}

// Zeros between the two halves of every staged sequence of the thread's
// fields (orders M .. N - M).
template <int P>
__device__ __forceinline__ void c2r45_zero_gap(float2 *bufs, int by, int nlat, int M, bool field_ok,
                                               int tid = threadIdx.x) {
  constexpr int N = kQ * P;
  constexpr int NPAIR = kThreads / P / kFB;
  constexpr int BUF = seq_pitch<P>();
  constexpr int kPairs = kFB / 2;
  constexpr int kMStep = kThreads / kPairs;
  const int Kh = (nlat + 1) / 2;
  const int f2 = tid % kPairs, m0 = tid / kPairs;
  const int fa = 2 * f2;
#pragma unroll 1
  for (int pq = 0; pq < NPAIR; pq++) {
    const int kq = by * NPAIR + pq;
    if (kq >= Kh || !field_ok) continue;
    float2 *Ba = bufs + (pq * kFB + fa) * BUF;
    for (int q = M + m0; q <= N - M; q += kMStep) {
      Ba[q] = make_float2(0.f, 0.f);
      Ba[BUF + q] = make_float2(0.f, 0.f);
    }
  }
}

// The synthesis proper, after staging (and a CTA barrier): every sequence
// buffer of `bufs` holds conj(Z); the inverse DFT is evaluated as
// conj(FFT(conj Z)), and the two real rows are written.
template <int P>
__device__ __forceinline__ void c2r45_synth(int bx, int by, float2 *bufs, const float2 *tw, float *__restrict__ y,
                                            int nlat, int B, int tid = threadIdx.x) {
  constexpr int N = kQ * P;
  constexpr int NPAIR = kThreads / P / kFB;
  constexpr int BUF = seq_pitch<P>();
  const int Kh = (nlat + 1) / 2;
  const int s = tid / P, t = tid % P;
  const int f = s % kFB, pp = s / kFB;
  const int b = bx * kFB + f;
  const int kp = by * NPAIR + pp;
  const int ksth = nlat - 1 - kp;
  const bool live = (b < B) && (kp < Kh);
  float2 *buf = bufs + s * BUF;
  float2 v[kQ];
#pragma unroll
  for (int j = 0; j < kQ; j++) v[j] = live ? buf[t + P * j] : make_float2(0.f, 0.f);
  __syncwarp();
  seq_fft<P>(v, t, buf, tw);
  if (!live) return;
  const bool eq = (kp == ksth);
  float *rn = y + ((int64_t)b * nlat + kp) * N;
  float *rs = y + ((int64_t)b * nlat + ksth) * N;
  int r = t, q = 0;  // j = 45 q + r
#pragma unroll 5
  for (int j = t; j < N; j += P) {
    const float2 o = buf[r * rpitch<P>() + q];
    rn[j] = o.x;
    if (!eq) rs[j] = -o.y;
    r += P;
    if (r >= kQ) {
      r -= kQ;
      q++;
    }
  }
}

template <int P, int kBatch>
__device__ __forceinline__ void c2r45_body(int bx, int by, const float *__restrict__ Gw, float *__restrict__ y,
                                           int nlat, int M, int B, FoldLayout fl, const float2 *__restrict__ twiddle,
                                           const float *__restrict__ ring_scale, int inverse_weights) {
  constexpr int N = kQ * P;
  constexpr int NPAIR = kThreads / P / kFB;
  constexpr int BUF = seq_pitch<P>();
  extern __shared__ float2 smem[];
  float2 *tw = smem;
  float2 *bufs = smem + N;
  const int Kh = (nlat + 1) / 2;
  const int b0 = bx * kFB;
  load_twiddles<P>(tw, twiddle);
  // stage conj(Z) in every sequence buffer; thread (f2, m0) stages fields
  // 2 f2 and 2 f2 + 1 (one 16-byte load per row), orders m0, m0 + 64, ...,
  // kBatch loads in flight (12: all of a thread's orders at nlon = 1440 in
  // one memory round trip; the grouped kernel, which holds every P's body,
  // keeps 6 to stay unspilled)
  constexpr int kPairs = kFB / 2;
  constexpr int kMStep = kThreads / kPairs;  // 64
  const int f2 = threadIdx.x % kPairs, m0 = threadIdx.x / kPairs;
  const int fa = 2 * f2;
  // fields past B stage zeros (their sequences are not synthesised)
  const bool field_ok = b0 + fa < B;
  const bool two = b0 + fa + 1 < B;
  const int64_t col = fold_col(fl, 2 * (int64_t)(b0 + fa));  // 4 columns of one 16-column group
  const int64_t pstride = fl.sp;                            // E row -> O row
  // the thread's items (ring pair pq, order m0 + i kMStep) in batches that
  // may span ring pairs, so that short rows (small grids, several ring
  // pairs per CTA) still keep kBatch loads in flight
  const int per = m0 < M ? (M - m0 + kMStep - 1) / kMStep : 0;
  const int total = field_ok ? NPAIR * per : 0;
  for (int it0 = 0; it0 < total; it0 += kBatch) {
    float4 ge[kBatch], go[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; u++) {
      ge[u] = go[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      const int it = it0 + u;
      if (it >= total) continue;
      const int pq = NPAIR == 1 ? 0 : it / per;
      const int m = m0 + (it - pq * per) * kMStep, kq = by * NPAIR + pq;
      if (kq >= Kh) continue;
      const float *g = Gw + fold_row(fl, m, 0, kq) + col;
      if (two) {
        ge[u] = *reinterpret_cast<const float4 *>(g);
        go[u] = *reinterpret_cast<const float4 *>(g + pstride);
      } else {
        const float2 a = *reinterpret_cast<const float2 *>(g), c = *reinterpret_cast<const float2 *>(g + pstride);
        ge[u] = make_float4(a.x, a.y, 0.f, 0.f);
        go[u] = make_float4(c.x, c.y, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int u = 0; u < kBatch; u++) {
      const int it = it0 + u;
      if (it >= total) break;
      const int pq = NPAIR == 1 ? 0 : it / per;
      const int m = m0 + (it - pq * per) * kMStep, kq = by * NPAIR + pq;
      if (kq >= Kh) continue;
      c2r45_put<P>(bufs + (pq * kFB + fa) * BUF, ge[u], go[u], m, kq, nlat, ring_scale, inverse_weights);
    }
  }
  c2r45_zero_gap<P>(bufs, by, nlat, M, field_ok);
  __syncthreads();
  c2r45_synth<P>(bx, by, bufs, tw, y, nlat, B);
}

template <int P>
__global__ void __launch_bounds__(kThreads, 2)
c2r45_kernel(const float *__restrict__ Gw, float *__restrict__ y, int nlat, int M, int B, FoldLayout fl,
             const float2 *__restrict__ twiddle, const float *__restrict__ ring_scale, int inverse_weights) {
  c2r45_body<P, 12>(blockIdx.x, blockIdx.y, Gw, y, nlat, M, B, fl, twiddle, ring_scale, inverse_weights);
}

// ---------------------------------------------------------------------------
// Persistent forms, one CTA per SM: the CTA walks the tiles (bx, by) of the
// grid above (tile = by gx + bx) in steps of the grid size, and the input of
// its next tile arrives in shared memory by asynchronous bulk copies while
// the current tile is transformed, so that DRAM and the FFT's instruction
// stream overlap inside every SM.  Every wait is bounded: a copy that does
// not arrive within the limit records SHT's timeout code in *err, and the
// CTA waits a little longer for what it still has in flight and returns.

// Analysis: two stages of NSEQ sequence buffers.  A stage first receives the
// tile's rows by bulk copies (sequence s: its northern row at float 0, its
// southern row at float N of the buffer; 2 N floats = N float2 <= BUF), is
// then read into registers by the sequence's lanes, and serves as the
// sequence buffers of that tile's FFT and output stage.  Two warp groups
// share the CTA (512 threads): the FFT group (warps 0-7, one sequence each)
// transforms tile i + 1 while the output group (warps 8-15) separates,
// folds and stores tile i from the other stage; mbarriers hand a stage from
// the copies to the FFT group (full), to the output group (fftd) and back
// to the copies of tile i + 2 (freed), which one output thread issues.
template <int P>
__host__ __device__ constexpr size_t r2c_pipe_smem() {
  return 64 + sizeof(float2) * ((size_t)kQ * P + 2 * (size_t)(kThreads / P) * seq_pitch<P>());
}

constexpr int kWsThreads = 2 * kThreads;

template <int P, class Out>
__global__ void __launch_bounds__(kWsThreads, 1)
r2c45_pipe_kernel(const float *__restrict__ x, Out out, int nlat, int M, int B, FoldLayout fl,
                  const float2 *__restrict__ twiddle, const float *__restrict__ ring_scale, int inverse_weights,
                  unsigned *err) {
  constexpr int N = kQ * P;
  constexpr int NPAIR = kThreads / P / kFB;
  constexpr int BUF = seq_pitch<P>();
  constexpr int NSEQ = kThreads / P;
  constexpr int kGroupWarps = kThreads / 32;
  constexpr uint32_t kRowBytes = 4u * N;
  extern __shared__ __align__(1024) unsigned char pipe_smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(pipe_smem);  // [2]
  uint64_t *fftd = full + 2, *freed = full + 4;                // [2] each
  float2 *tw = reinterpret_cast<float2 *>(pipe_smem + 64);
  float2 *stage0 = tw + N;
  const int Kh = (nlat + 1) / 2;
  const int gx = (B + kFB - 1) / kFB;
  const int ntiles = gx * ((Kh + NPAIR - 1) / NPAIR);
  const int lane = threadIdx.x & 31;
  const bool fft_group = threadIdx.x < kThreads;
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    for (int q = 0; q < 2; q++) {
      tc::mbar_init(&full[q], 1);
      tc::mbar_init(&fftd[q], kGroupWarps);
      tc::mbar_init(&freed[q], kGroupWarps);
    }
    tc::mbar_fence_init();
  }
  if (fft_group) load_twiddles<P>(tw, twiddle);
  __syncthreads();
  if (fft_group) {
    const int s = threadIdx.x / P, t = threadIdx.x % P;
    const int f = s % kFB, pp = s / kFB;
    int i = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += G, i++) {
      const int st = i & 1;
      // a warp leaves together (it meets at warp barriers below)
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&full[st], (i >> 1) & 1, err))) break;
      const int bx = tile % gx, by = tile / gx;
      float2 *buf = stage0 + (st * NSEQ + s) * BUF;
      const int b = bx * kFB + f, kp = by * NPAIR + pp;
      const bool live = (b < B) && (kp < Kh);
      const bool eq = kp == nlat - 1 - kp;
      const float *rn = reinterpret_cast<const float *>(buf), *rs = rn + N;
      float2 v[kQ];
#pragma unroll
      for (int j = 0; j < kQ; j++)
        v[j] = live ? make_float2(rn[t + P * j], eq ? 0.f : rs[t + P * j]) : make_float2(0.f, 0.f);
      __syncwarp();
      seq_fft<P>(v, t, buf, tw);
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&fftd[st]);
    }
  } else {
    const int et = threadIdx.x - kThreads;
    const bool producer = et < 32;  // the output group's first warp issues the copies
    // the copies of tile `tile` into stage `st`: lane j of the producer warp
    // copies the rows of sequences j, j + 32, ...; lane 0 announces the bytes
    int last_par[2] = {-1, -1};
    auto issue = [&](int tile, int st, int par) {
      const int bx = tile % gx, by = tile / gx;
      float2 *sb = stage0 + st * NSEQ * BUF;
      uint32_t bytes = 0;
      for (int q = lane; q < NSEQ; q += 32) {
        const int b = bx * kFB + q % kFB, kp = by * NPAIR + q / kFB;
        if (b < B && kp < Kh) bytes += (kp == nlat - 1 - kp ? 1u : 2u) * kRowBytes;
      }
      bytes = __reduce_add_sync(0xffffffffu, bytes);
      if (lane == 0) tc::mbar_arrive_expect_tx(&full[st], bytes);
      __syncwarp();
      for (int q = lane; q < NSEQ; q += 32) {
        const int b = bx * kFB + q % kFB, kp = by * NPAIR + q / kFB, ks = nlat - 1 - kp;
        if (b >= B || kp >= Kh) continue;
        float *dst = reinterpret_cast<float *>(sb + q * BUF);
        tc::bulk_load(dst, x + ((int64_t)b * nlat + kp) * N, kRowBytes, &full[st]);
        if (ks != kp) tc::bulk_load(dst + N, x + ((int64_t)b * nlat + ks) * N, kRowBytes, &full[st]);
      }
      last_par[st] = par;
    };
    if (producer) {
      if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0, 0);
      if ((int)blockIdx.x + G < ntiles) issue(blockIdx.x + G, 1, 0);
    }
    int i = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += G, i++) {
      const int st = i & 1;
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&fftd[st], (i >> 1) & 1, err))) break;
      const int bx = tile % gx, by = tile / gx;
      r2c45_emit<P, Out>(bx, by, stage0 + st * NSEQ * BUF, out, nlat, M, B, fl, ring_scale, inverse_weights, et);
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&freed[st]);
      if (producer && tile + 2 * G < ntiles) {
        // the warp leaves together: its lanes issue the copies together
        if (!__all_sync(0xffffffffu, tc::mbar_wait(&freed[st], (i >> 1) & 1, err))) break;
        issue(tile + 2 * G, st, ((i >> 1) + 1) & 1);
      }
    }
    // copies still in flight (a wait gave up): let them land (bounded)
    if (et == 0)
      for (int q = 0; q < 2; q++)
        if (last_par[q] >= 0) tc::mbar_wait(&full[q], (uint32_t)last_par[q], nullptr, 100000000ull);
  }
}

// Synthesis: one staging buffer of the tile's folded rows, [NPAIR][nrows]
// rows of 32 floats (E and O of the tile's 8 fields at one order m: the
// parity-paired layout keeps them in one 128-byte segment), filled by TMA
// boxes of box_rows orders.  The CTA turns it into conj(Z) in the sequence
// buffers, after which the next tile's boxes are issued into it while this
// tile's FFTs and row stores run.
template <int P>
size_t c2r_pipe_smem(int nrows) {
  return (size_t)(kThreads / P / kFB) * nrows * 128 + 16 + sizeof(float2) * ((size_t)kQ * P +
                                                                            (size_t)(kThreads / P) * seq_pitch<P>());
}

template <int P>
__global__ void __launch_bounds__(kThreads, 1)
c2r45_pipe_kernel(const __grid_constant__ CUtensorMap gmap, float *__restrict__ y, int nlat, int M, int B,
                  int box_rows, int nbox, const float2 *__restrict__ twiddle, const float *__restrict__ ring_scale,
                  int inverse_weights, unsigned *err) {
  constexpr int N = kQ * P;
  constexpr int NPAIR = kThreads / P / kFB;
  constexpr int BUF = seq_pitch<P>();
  constexpr int kPairs = kFB / 2;
  constexpr int kMStep = kThreads / kPairs;  // 64
  extern __shared__ __align__(1024) unsigned char pipe_smem[];
  const int nrows = nbox * box_rows;
  float *stg = reinterpret_cast<float *>(pipe_smem);
  uint64_t *bar = reinterpret_cast<uint64_t *>(pipe_smem + (size_t)NPAIR * nrows * 128);
  float2 *tw = reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(bar) + 16);
  float2 *bufs = tw + N;
  const int Kh = (nlat + 1) / 2;
  const int gx = (B + kFB - 1) / kFB;
  const int ntiles = gx * ((Kh + NPAIR - 1) / NPAIR);
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    tc::tma_prefetch_desc(&gmap);
    tc::mbar_init(bar, 1);
    tc::mbar_fence_init();
  }
  load_twiddles<P>(tw, twiddle);
  __syncthreads();
  auto issue = [&](int tile) {
    const int bx = tile % gx, by = tile / gx;
    int live = 0;
    for (int pq = 0; pq < NPAIR; pq++) live += (by * NPAIR + pq < Kh);
    tc::mbar_arrive_expect_tx(bar, (uint32_t)(live * nrows * 128));
    for (int pq = 0; pq < NPAIR; pq++) {
      const int kq = by * NPAIR + pq;
      if (kq >= Kh) continue;
      for (int j = 0; j < nbox; j++)
        tc::tma_load_3d(stg + ((size_t)pq * nrows + (size_t)j * box_rows) * 32, &gmap, bar, 32 * bx, kq,
                        j * box_rows);
    }
  };
  if (threadIdx.x == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x);
  const int f2 = threadIdx.x % kPairs, m0 = threadIdx.x / kPairs;
  const int fa = 2 * f2;
  int i = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += G, i++) {
    const bool ok = tc::mbar_wait(bar, i & 1, err);
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) tc::mbar_wait(bar, i & 1, nullptr, 100000000ull);
      __syncthreads();
      return;
    }
    const int bx = tile % gx, by = tile / gx;
    const int b0 = bx * kFB;
    const bool field_ok = b0 + fa < B;
    const bool two = b0 + fa + 1 < B;
    if (field_ok) {
#pragma unroll 1
      for (int pq = 0; pq < NPAIR; pq++) {
        const int kq = by * NPAIR + pq;
        if (kq >= Kh) continue;
        const float *row = stg + (size_t)pq * nrows * 32 + 4 * f2;
        float2 *Ba = bufs + (pq * kFB + fa) * BUF;
#pragma unroll 4
        for (int m = m0; m < M; m += kMStep) {
          float4 ge = *reinterpret_cast<const float4 *>(row + m * 32);
          float4 go = *reinterpret_cast<const float4 *>(row + m * 32 + 16);
          if (!two) {
            ge.z = ge.w = 0.f;
            go.z = go.w = 0.f;
          }
          c2r45_put<P>(Ba, ge, go, m, kq, nlat, ring_scale, inverse_weights);
        }
      }
    }
    c2r45_zero_gap<P>(bufs, by, nlat, M, field_ok);
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0 && tile + G < ntiles) issue(tile + G);
    c2r45_synth<P>(bx, by, bufs, tw, y, nlat, B);
    __syncthreads();
  }
}

// Synthesis, warp-specialised (nlon = 45 P, P >= 8): two stages of NSEQ
// sequence buffers, each first filled by the tile's TMA boxes (the staged
// rows, [NPAIR][nrows][32 floats], fit in the sequence buffers) and then
// turned into conj(Z) in place: the conversion group (warps 0-7) reads all
// its staged items into registers, meets at a named barrier, and writes the
// sequences over them; the FFT group (warps 8-15) transforms and stores the
// tile of the other stage meanwhile.  mbarriers hand a stage from the boxes
// to the conversion group (full), to the FFT group (conv) and back to the
// boxes of the tile after next (freed, which one FFT thread waits for
// before it issues them).
constexpr int kC2rItems = 12;  // a thread's (ring pair, order) items: NPAIR x ceil(M / 64) for P >= 8

// AND of v over the `count` threads of named barrier `id` (a barrier too).
template <int id, int count>
__device__ __forceinline__ bool group_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.and.pred p, %2, %3, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"(v ? 1u : 0u), "n"(id), "n"(count)
      : "memory");
  return r != 0;
}

template <int P>
__host__ __device__ constexpr size_t c2r_ws_stage_bytes() {
  return sizeof(float2) * (size_t)(kThreads / P) * seq_pitch<P>();
}
template <int P>
size_t c2r_ws_smem() {
  return 2 * c2r_ws_stage_bytes<P>() + 64 + sizeof(float2) * (size_t)kQ * P;
}

template <int P>
__global__ void __launch_bounds__(kWsThreads, 1)
c2r45_ws_kernel(const __grid_constant__ CUtensorMap gmap, float *__restrict__ y, int nlat, int M, int B,
                int box_rows, int nbox, const float2 *__restrict__ twiddle, const float *__restrict__ ring_scale,
                int inverse_weights, unsigned *err) {
  static_assert(P >= 8, "the conversion keeps at most kC2rItems items per thread");
  constexpr int NPAIR = kThreads / P / kFB;
  constexpr int BUF = seq_pitch<P>();
  constexpr int kPairs = kFB / 2;
  constexpr int kMStep = kThreads / kPairs;  // 64
  constexpr int kGroupWarps = kThreads / 32;
  constexpr size_t kStage = c2r_ws_stage_bytes<P>();
  extern __shared__ __align__(1024) unsigned char pipe_smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(pipe_smem + 2 * kStage);  // [2]
  uint64_t *conv = full + 2, *freed = full + 4;
  float2 *tw = reinterpret_cast<float2 *>(pipe_smem + 2 * kStage + 64);
  const int nrows = nbox * box_rows;
  const int Kh = (nlat + 1) / 2;
  const int gx = (B + kFB - 1) / kFB;
  const int ntiles = gx * ((Kh + NPAIR - 1) / NPAIR);
  const int lane = threadIdx.x & 31;
  const int G = gridDim.x;
  auto stage = [&](int st) { return pipe_smem + (size_t)st * kStage; };
  if (threadIdx.x == 0) {
    tc::tma_prefetch_desc(&gmap);
    for (int q = 0; q < 2; q++) {
      tc::mbar_init(&full[q], 1);
      tc::mbar_init(&conv[q], kGroupWarps);
      tc::mbar_init(&freed[q], kGroupWarps);
    }
    tc::mbar_fence_init();
  }
  if (threadIdx.x < kThreads) load_twiddles<P>(tw, twiddle);
  __syncthreads();
  if (threadIdx.x < kThreads) {
    // conversion group
    const int f2 = threadIdx.x % kPairs, m0 = threadIdx.x / kPairs;
    const int fa = 2 * f2;
    int i = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += G, i++) {
      const int st = i & 1;
      // the group leaves together (it meets at named barriers below)
      if (!group_all<2, kThreads>(tc::mbar_wait(&full[st], (i >> 1) & 1, err))) break;
      const int bx = tile % gx, by = tile / gx;
      const int b0 = bx * kFB;
      const bool field_ok = b0 + fa < B;
      const bool two = b0 + fa + 1 < B;
      const float *stg = reinterpret_cast<const float *>(stage(st));
      float4 ge[kC2rItems], go[kC2rItems];
      int u = 0;
#pragma unroll
      for (int pq = 0; pq < NPAIR; pq++) {
#pragma unroll
        for (int k = 0; k < kC2rItems / NPAIR; k++, u++) {
          const int m = m0 + k * kMStep;
          ge[u] = go[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (field_ok && m < M && by * NPAIR + pq < Kh) {
            const float *row = stg + ((size_t)pq * nrows + m) * 32 + 4 * f2;
            ge[u] = *reinterpret_cast<const float4 *>(row);
            go[u] = *reinterpret_cast<const float4 *>(row + 16);
            if (!two) {
              ge[u].z = ge[u].w = 0.f;
              go[u].z = go[u].w = 0.f;
            }
          }
        }
      }
      // every staged item of the stage is in registers: write over them
      asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory");
      float2 *bufs = reinterpret_cast<float2 *>(stage(st));
      u = 0;
#pragma unroll
      for (int pq = 0; pq < NPAIR; pq++) {
        const int kq = by * NPAIR + pq;
#pragma unroll
        for (int k = 0; k < kC2rItems / NPAIR; k++, u++) {
          const int m = m0 + k * kMStep;
          if (field_ok && m < M && kq < Kh)
            c2r45_put<P>(bufs + (pq * kFB + fa) * BUF, ge[u], go[u], m, kq, nlat, ring_scale, inverse_weights);
        }
      }
      c2r45_zero_gap<P>(bufs, by, nlat, M, field_ok, threadIdx.x);
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&conv[st]);
    }
  } else {
    // FFT group; thread 0 of the group issues the boxes
    const int bt = threadIdx.x - kThreads;
    int last_par[2] = {-1, -1};
    auto issue = [&](int tile, int st, int par) {
      const int bx = tile % gx, by = tile / gx;
      int live = 0;
      for (int pq = 0; pq < NPAIR; pq++) live += (by * NPAIR + pq < Kh);
      tc::mbar_arrive_expect_tx(&full[st], (uint32_t)(live * nrows * 128));
      float *stg = reinterpret_cast<float *>(stage(st));
      for (int pq = 0; pq < NPAIR; pq++) {
        const int kq = by * NPAIR + pq;
        if (kq >= Kh) continue;
        for (int j = 0; j < nbox; j++)
          tc::tma_load_3d(stg + ((size_t)pq * nrows + (size_t)j * box_rows) * 32, &gmap, &full[st], 32 * bx, kq,
                          j * box_rows);
      }
      last_par[st] = par;
    };
    if (bt == 0) {
      if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0, 0);
      if ((int)blockIdx.x + G < ntiles) issue(blockIdx.x + G, 1, 0);
    }
    int i = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += G, i++) {
      const int st = i & 1;
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&conv[st], (i >> 1) & 1, err))) break;
      const int bx = tile % gx, by = tile / gx;
      c2r45_synth<P>(bx, by, reinterpret_cast<float2 *>(stage(st)), tw, y, nlat, B, bt);
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&freed[st]);
      if (bt == 0 && tile + 2 * G < ntiles) {
        if (!tc::mbar_wait(&freed[st], (i >> 1) & 1, err)) break;
        issue(tile + 2 * G, st, ((i >> 1) + 1) & 1);
      }
    }
    if (bt == 0)
      for (int q = 0; q < 2; q++)
        if (last_par[q] >= 0) tc::mbar_wait(&full[q], (uint32_t)last_par[q], nullptr, 100000000ull);
  }
}

// Grouped launches: one grid over several problems (grids and batches) of
// one batched call.  CTA j belongs to the segment s with blk0[s] <= j <
// blk0[s + 1]; its (bx, by) follow from gx[s], and the segment's P selects
// the transform length.
struct Fft45Seg {
  const float *in;
  float *outf;
  __nv_bfloat16 *hi, *lo;
  const float2 *tw;
  const float *ring;
  FoldLayout fl;
  int nlat, M, B, wts, P, gx, blk0;
};
struct Fft45Group {
  Fft45Seg seg[kMaxFftGroup];
  int nseg;
};

__device__ __forceinline__ int group_segment(const Fft45Group &g, int blk) {
  int s = 0;
  while (s + 1 < g.nseg && blk >= g.seg[s + 1].blk0) s++;
  return s;
}

template <bool kBF16>
__global__ void __launch_bounds__(kThreads, 2) r2c45_grouped_kernel(const __grid_constant__ Fft45Group g) {
  const int s = group_segment(g, blockIdx.x);
  const Fft45Seg &q = g.seg[s];
  const int local = blockIdx.x - q.blk0;
  const int bx = local % q.gx, by = local / q.gx;
  if (kBF16) {
    const OutBF16 out{q.hi, q.lo};
    switch (q.P) {
      case 32: r2c45_body<32>(bx, by, q.in, out, q.nlat, q.M, q.B, q.fl, q.tw, q.ring, q.wts); break;
      case 16: r2c45_body<16>(bx, by, q.in, out, q.nlat, q.M, q.B, q.fl, q.tw, q.ring, q.wts); break;
      case 8: r2c45_body<8>(bx, by, q.in, out, q.nlat, q.M, q.B, q.fl, q.tw, q.ring, q.wts); break;
      default: r2c45_body<4>(bx, by, q.in, out, q.nlat, q.M, q.B, q.fl, q.tw, q.ring, q.wts); break;
    }
  } else {
    const OutF32 out{q.outf};
    switch (q.P) {
      case 32: r2c45_body<32>(bx, by, q.in, out, q.nlat, q.M, q.B, q.fl, q.tw, q.ring, q.wts); break;
      case 16: r2c45_body<16>(bx, by, q.in, out, q.nlat, q.M, q.B, q.fl, q.tw, q.ring, q.wts); break;
      case 8: r2c45_body<8>(bx, by, q.in, out, q.nlat, q.M, q.B, q.fl, q.tw, q.ring, q.wts); break;
      default: r2c45_body<4>(bx, by, q.in, out, q.nlat, q.M, q.B, q.fl, q.tw, q.ring, q.wts); break;
    }
  }
}

__global__ void __launch_bounds__(kThreads, 2) c2r45_grouped_kernel(const __grid_constant__ Fft45Group g) {
  const int s = group_segment(g, blockIdx.x);
  const Fft45Seg &q = g.seg[s];
  const int local = blockIdx.x - q.blk0;
  const int bx = local % q.gx, by = local / q.gx;
  switch (q.P) {
    case 32: c2r45_body<32, 6>(bx, by, q.in, q.outf, q.nlat, q.M, q.B, q.fl, q.tw, q.ring, q.wts); break;
    case 16: c2r45_body<16, 6>(bx, by, q.in, q.outf, q.nlat, q.M, q.B, q.fl, q.tw, q.ring, q.wts); break;
    case 8: c2r45_body<8, 6>(bx, by, q.in, q.outf, q.nlat, q.M, q.B, q.fl, q.tw, q.ring, q.wts); break;
    default: c2r45_body<4, 6>(bx, by, q.in, q.outf, q.nlat, q.M, q.B, q.fl, q.tw, q.ring, q.wts); break;
  }
}

template <int P>
size_t smem45() {
  return sizeof(float2) * ((size_t)kQ * P + (size_t)(kThreads / P) * seq_pitch<P>());
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int max_smem_optin() {
  static int v = 0;
  if (v == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) v = 0;
  }
  return v;
}

template <int P, class Out>
cudaError_t r2c45(const float *x, Out out, int nlat, int M, int B, FoldLayout fl, const float2 *tw, const float *ring,
                  int wts, cudaStream_t st, unsigned *err) {
  const int Kh = (nlat + 1) / 2;
  constexpr int NPAIR = kThreads / P / kFB;
  dim3 grid((B + kFB - 1) / kFB, (Kh + NPAIR - 1) / NPAIR);
  cudaError_t e;
  constexpr size_t psmem = r2c_pipe_smem<P>();
  // persistent warp-specialised form (the rows arrive by 16-byte-aligned
  // bulk copies) at nlon = 360, 720 and 1440; at nlon = 180 (128 short rows
  // per tile) the non-persistent kernel is faster (measured per grid)
  if (P >= 8 && aligned16(x) && psmem <= (size_t)max_smem_optin()) {
    e = cudaFuncSetAttribute((const void *)r2c45_pipe_kernel<P, Out>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)psmem);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (int64_t)grid.x * grid.y;
    const unsigned g = (unsigned)std::min<int64_t>(ntiles, sm_count());
    r2c45_pipe_kernel<P, Out><<<g, kWsThreads, psmem, st>>>(x, out, nlat, M, B, fl, tw, ring, wts, err);
    return cudaGetLastError();
  }
  const size_t smem = smem45<P>();
  e = cudaFuncSetAttribute((const void *)r2c45_kernel<P, Out>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  r2c45_kernel<P, Out><<<grid, kThreads, smem, st>>>(x, out, nlat, M, B, fl, tw, ring, wts);
  return cudaGetLastError();
}

template <int P>
cudaError_t c2r45(const float *G, float *y, int nlat, int M, int B, FoldLayout fl, const float2 *tw, const float *ring,
                  int wts, cudaStream_t st, unsigned *err) {
  const int Kh = (nlat + 1) / 2;
  constexpr int NPAIR = kThreads / P / kFB;
  dim3 grid((B + kFB - 1) / kFB, (Kh + NPAIR - 1) / NPAIR);
  cudaError_t e;
  if (fl.cg && aligned16(G) && M >= 1) {
    // persistent form on the parity-paired layout: TMA boxes of box_rows
    // orders of one ring pair and one 8-field group (128 bytes per order)
    const int nbox = (M + 255) / 256, box_rows = (M + nbox - 1) / nbox;
    const size_t psmem = c2r_pipe_smem<P>(nbox * box_rows);
    CUtensorMap gm;
    const bool ws = P >= 8 && (size_t)NPAIR * nbox * box_rows * 128 <= c2r_ws_stage_bytes<P>() &&
                    c2r_ws_smem<P>() <= (size_t)max_smem_optin();
    if (ws && tc_encode_pair_rows_f32(&gm, G, fl, Kh, M, box_rows)) {
      // warp-specialised: conversion and FFT groups on two stages
      const size_t wsmem = c2r_ws_smem<P>();
      e = cudaFuncSetAttribute((const void *)c2r45_ws_kernel<P < 8 ? 8 : P>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem);
      if (e != cudaSuccess) return e;
      const int64_t ntiles = (int64_t)grid.x * grid.y;
      const unsigned g = (unsigned)std::min<int64_t>(ntiles, sm_count());
      c2r45_ws_kernel<P < 8 ? 8 : P><<<g, kWsThreads, wsmem, st>>>(gm, y, nlat, M, B, box_rows, nbox, tw, ring, wts,
                                                                      err);
      return cudaGetLastError();
    }
    if (psmem <= (size_t)max_smem_optin() && tc_encode_pair_rows_f32(&gm, G, fl, Kh, M, box_rows)) {
      e = cudaFuncSetAttribute((const void *)c2r45_pipe_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)psmem);
      if (e != cudaSuccess) return e;
      const int64_t ntiles = (int64_t)grid.x * grid.y;
      const unsigned g = (unsigned)std::min<int64_t>(ntiles, sm_count());
      c2r45_pipe_kernel<P><<<g, kThreads, psmem, st>>>(gm, y, nlat, M, B, box_rows, nbox, tw, ring, wts, err);
      return cudaGetLastError();
    }
  }
  const size_t smem = smem45<P>();
  e = cudaFuncSetAttribute((const void *)c2r45_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  c2r45_kernel<P><<<grid, kThreads, smem, st>>>(G, y, nlat, M, B, fl, tw, ring, wts);
  return cudaGetLastError();
}

template <class Out>
cudaError_t r2c45_dispatch(int nlon, const float *x, Out out, int nlat, int M, int B, FoldLayout fl, const float2 *tw,
                           const float *ring, int wts, cudaStream_t st, unsigned *err) {
  switch (nlon / kQ) {
    case 32: return r2c45<32>(x, out, nlat, M, B, fl, tw, ring, wts, st, err);
    case 16: return r2c45<16>(x, out, nlat, M, B, fl, tw, ring, wts, st, err);
    case 8: return r2c45<8>(x, out, nlat, M, B, fl, tw, ring, wts, st, err);
    default: return r2c45<4>(x, out, nlat, M, B, fl, tw, ring, wts, st, err);
  }
}

size_t smem45_of(int P) {
  switch (P) {
    case 32: return smem45<32>();
    case 16: return smem45<16>();
    case 8: return smem45<8>();
    default: return smem45<4>();
  }
}

// Fill the CTA ranges of a group; returns the total CTA count and the
// largest shared-memory size.
int64_t group_layout(Fft45Group &g, const Fft45Item *items, int n, size_t &smem) {
  g.nseg = n;
  int64_t blk = 0;
  smem = 0;
  for (int i = 0; i < n; i++) {
    const Fft45Item &it = items[i];
    Fft45Seg &q = g.seg[i];
    const int P = it.nlon / kQ;
    const int NPAIR = kThreads / P / kFB;
    const int Kh = (it.nlat + 1) / 2;
    q.in = it.in;
    q.outf = it.outf;
    q.hi = it.hi;
    q.lo = it.lo;
    q.tw = it.twiddle;
    q.ring = it.ring_scale;
    q.nlat = it.nlat;
    q.M = it.M;
    q.B = it.B;
    q.fl = it.fl;
    q.wts = it.inverse_weights;
    q.P = P;
    q.gx = (it.B + kFB - 1) / kFB;
    q.blk0 = (int)blk;
    blk += (int64_t)q.gx * ((Kh + NPAIR - 1) / NPAIR);
    smem = std::max(smem, smem45_of(P));
  }
  return blk;
}

}  // namespace

cudaError_t launch_r2c45_grouped(const Fft45Item *items, int n, bool bf16, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > kMaxFftGroup) return cudaErrorInvalidValue;
  for (int i = 0; i < n; i++)
    if (!fft45_supported(items[i].nlon) || items[i].B <= 0) return cudaErrorInvalidValue;
  Fft45Group g{};
  size_t smem = 0;
  const int64_t blocks = group_layout(g, items, n, smem);
  if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
  const void *fn = bf16 ? (const void *)r2c45_grouped_kernel<true> : (const void *)r2c45_grouped_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (bf16)
    r2c45_grouped_kernel<true><<<(unsigned)blocks, kThreads, smem, st>>>(g);
  else
    r2c45_grouped_kernel<false><<<(unsigned)blocks, kThreads, smem, st>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_c2r45_grouped(const Fft45Item *items, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > kMaxFftGroup) return cudaErrorInvalidValue;
  for (int i = 0; i < n; i++)
    if (!fft45_supported(items[i].nlon) || items[i].B <= 0) return cudaErrorInvalidValue;
  Fft45Group g{};
  size_t smem = 0;
  const int64_t blocks = group_layout(g, items, n, smem);
  if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute((const void *)c2r45_grouped_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  c2r45_grouped_kernel<<<(unsigned)blocks, kThreads, smem, st>>>(g);
  return cudaGetLastError();
}

bool fft45_supported(int nlon) {
  return nlon == 45 * 32 || nlon == 45 * 16 || nlon == 45 * 8 || nlon == 45 * 4;
}

cudaError_t launch_r2c45(const float *x, float *Fw, __nv_bfloat16 *Fhi, __nv_bfloat16 *Flo, int nlat, int nlon,
                         int M, int B, FoldLayout fl, const float2 *twiddle, const float *ring_scale, int inverse_weights,
                         cudaStream_t st, unsigned *err) {
  if (B <= 0) return cudaSuccess;
  if (Fw) return r2c45_dispatch(nlon, x, OutF32{Fw}, nlat, M, B, fl, twiddle, ring_scale, inverse_weights, st, err);
  return r2c45_dispatch(nlon, x, OutBF16{Fhi, Flo}, nlat, M, B, fl, twiddle, ring_scale, inverse_weights, st, err);
}

cudaError_t launch_c2r45(const float *Gw, float *y, int nlat, int nlon, int M, int B, FoldLayout fl,
                         const float2 *twiddle, const float *ring_scale, int inverse_weights, cudaStream_t st,
                         unsigned *err) {
  if (B <= 0) return cudaSuccess;
  switch (nlon / kQ) {
    case 32: return c2r45<32>(Gw, y, nlat, M, B, fl, twiddle, ring_scale, inverse_weights, st, err);
    case 16: return c2r45<16>(Gw, y, nlat, M, B, fl, twiddle, ring_scale, inverse_weights, st, err);
    case 8: return c2r45<8>(Gw, y, nlat, M, B, fl, twiddle, ring_scale, inverse_weights, st, err);
    default: return c2r45<4>(Gw, y, nlat, M, B, fl, twiddle, ring_scale, inverse_weights, st, err);
  }
}

}  // namespace shtgb
