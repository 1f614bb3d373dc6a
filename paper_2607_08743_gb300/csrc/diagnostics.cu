// Analytic initial data generated on the device, the pi-symmetry monitor
// (Sec. 3.2) and the symmetrisation of data.
#include "sacrak_dev.cuh"

namespace sacrak {

// SplitMix64 output function (Steele, Lea & Flood 2014) applied to state x
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// uniform value in [-1, 1) of field f at level-global cell (i, j, k)
__device__ __forceinline__ double noise_value(uint64_t seed, int f, long long i, long long j,
                                              long long k) {
  uint64_t h = splitmix64(seed + (uint64_t)f);
  h = splitmix64(h ^ (uint64_t)i);
  h = splitmix64(h ^ (uint64_t)j);
  h = splitmix64(h ^ (uint64_t)k);
  return __dsub_rn(__dmul_rn(__dmul_rn((double)(h >> 11), 0x1.0p-53), 2.0), 1.0);
}

// Coordinates and arithmetic use explicitly rounded operations so that the
// values agree bit for bit with a plain left-to-right evaluation on the host.
__global__ void init_data_kernel(InitArgs A, int patch) {
  const DevPatch* P = A.patches + patch;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = (long long)P->NX * P->NY * P->NZ;
  if (id >= tot) return;
  const int I = id % P->NX, J = (id / P->NX) % P->NY, K = id / ((long long)P->NX * P->NY);
  const int idx[3] = {I, J, K};
  double x[3];
#pragma unroll
  for (int d = 0; d < 3; ++d)
    x[d] = __dadd_rn(P->origin[d], __dmul_rn((double)(idx[d] - GH) + 0.5, P->dx));
  double v[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) v[f] = flat_value(f);
  if (A.kind == 1) {
    double psi = 1.0;
    for (int a = 0; a < A.npunct; ++a) {
      double dx = __dsub_rn(x[0], A.pos[3 * a]);
      double dy = __dsub_rn(x[1], A.pos[3 * a + 1]);
      double dz = __dsub_rn(x[2], A.pos[3 * a + 2]);
      double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
      double r = __dsqrt_rn(r2);
      psi = __dadd_rn(psi, __ddiv_rn(A.m[a], __dmul_rn(2.0, r)));
    }
    double W = __ddiv_rn(1.0, __dmul_rn(psi, psi));
    v[F_W] = W;
    v[F_ALP] = W;
  } else if (A.kind == 2) {
    const double pi = 3.141592653589793;
    double ph = 2.0 * pi * x[0] / A.gw_len;
    double H = 1.0 - A.gw_amp * sin(ph);
    double dH = -A.gw_amp * cos(ph) * 2.0 * pi / A.gw_len;
    double Kxx = -(pi * A.gw_amp / A.gw_len) * cos(ph) / sqrt(H);
    double K = Kxx / H;
    double W = pow(H, -1.0 / 6.0);
    v[F_W] = W;
    v[F_GXX] = pow(H, 2.0 / 3.0);
    v[F_GYY] = pow(H, -1.0 / 3.0);
    v[F_GZZ] = v[F_GYY];
    v[F_KH] = K;
    v[F_AXX] = 2.0 / 3.0 * W * W * Kxx;
    v[F_AYY] = -1.0 / 3.0 * W * W * K;
    v[F_AZZ] = v[F_AYY];
    v[F_GAMX] = 2.0 / 3.0 * pow(H, -5.0 / 3.0) * dH;
    v[F_ALP] = sqrt(H);
  }
  const long long q = I + (long long)J * P->px + (long long)K * P->plane;
  double* u = P->buf[A.levels[P->level].ring];
  if (A.noise_amp != 0.0) {
    long long gi[3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
      gi[d] = (long long)llrint((P->origin[d] - A.lo[d]) / P->dx) + idx[d] - GH;
    for (int f = 0; f < NF; ++f)
      v[f] = __dadd_rn(v[f], __dmul_rn(A.noise_amp, noise_value(A.seed, f, gi[0], gi[1], gi[2])));
  }
  for (int f = 0; f < NF; ++f) u[f * P->fstride + q] = v[f];
}

// points with x < 0 (array index below NX/2 on a patch centred on x = y = 0)
// take the parity-signed value of their partner (-x, -y, z)
__global__ void symmetrise_kernel(const DevPatch* patches, const DevLevel* levels, int patch) {
  const DevPatch* P = patches + patch;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int half = P->NX / 2;
  const long long tot = (long long)half * P->NY * P->NZ;
  if (id >= tot) return;
  const int I = id % half, J = (id / half) % P->NY, K = id / ((long long)half * P->NY);
  double* u = P->buf[levels[P->level].ring];
  const long long q = I + (long long)J * P->px + (long long)K * P->plane;
  const long long qm = (P->NX - 1 - I) + (long long)(P->NY - 1 - J) * P->px + (long long)K * P->plane;
  for (int f = 0; f < NF; ++f) {
    double s = (double)pi_parity(f);
    u[f * P->fstride + q] = s * u[f * P->fstride + qm];
  }
}

// max |f - s_f f(mirror)| over all points and fields; block partial maxima
__global__ void pi_symmetry_kernel(const DevPatch* patches, const DevLevel* levels, int patch,
                                   double* partial) {
  __shared__ double red[8];
  const DevPatch* P = patches + patch;
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = (long long)P->NX * P->NY * P->NZ;
  double mx = 0.0;
  if (id < tot) {
    const int I = id % P->NX, J = (id / P->NX) % P->NY, K = id / ((long long)P->NX * P->NY);
    const double* u = P->buf[levels[P->level].ring];
    const long long q = I + (long long)J * P->px + (long long)K * P->plane;
    const long long qm =
        (P->NX - 1 - I) + (long long)(P->NY - 1 - J) * P->px + (long long)K * P->plane;
    for (int f = 0; f < NF; ++f) {
      double d = fabs(u[f * P->fstride + q] - (double)pi_parity(f) * u[f * P->fstride + qm]);
      if (!(d <= mx)) mx = isnan(d) ? INFINITY : d;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    partial[blockIdx.x] = m;
  }
}

__global__ void max_partials_kernel(const double* partial, int n, double* out) {
  __shared__ double sh[256];
  double m = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) m = fmax(m, partial[b]);
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

void launch_init(const InitArgs& a, int patch, long long tot, cudaStream_t st) {
  init_data_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, st>>>(a, patch);
}

void launch_symmetrise(const DevPatch* p, const DevLevel* l, int patch, long long half_tot,
                       cudaStream_t st) {
  symmetrise_kernel<<<(unsigned)((half_tot + 127) / 128), 128, 0, st>>>(p, l, patch);
}

int launch_pi_symmetry(const DevPatch* p, const DevLevel* l, int patch, long long tot,
                       double* partial, double* out, cudaStream_t st) {
  int nb = (int)((tot + 255) / 256);
  pi_symmetry_kernel<<<nb, 256, 0, st>>>(p, l, patch, partial);
  max_partials_kernel<<<1, 256, 0, st>>>(partial, nb, out);
  return nb;
}

// ---------------------------------------------------------------------------
// ADM mass, angular momentum (Sec. 2.3) and linear momentum (Sec. 3.2) on the
// coordinate sphere |x - c| = r, with the proper surface element
// dS_i = sqrt(g) n_i r^2 dOmega:
//   M   = 1/(16 pi) int g^ik g^jl (d_j g_kl - d_k g_jl) dS_i
//   J_z = 1/(8 pi)  int (x K_y^j - y K_x^j) dS_j
//   P_i = 1/(8 pi)  int (K_i^j - delta_i^j K) dS_j
// The integrands are formed at cell centres from g_ij = gt_ij / W^2 and
// K_ij = (At_ij + gt_ij K / 3) / W^2 (K = Khat + 2 Theta) with 4th-order
// centred derivatives, interpolated to the sphere with the 4 x 4 x 4 nearest
// cell centres (tricubic Lagrange), and integrated with Gauss-Legendre nodes
// in cos(theta) times the trapezoid rule in phi.  One block per theta ring;
// every sum runs in a fixed order.

// Integrands per coordinate area at array offset q: mass flux density m^i,
// kk[i][j] = sqrt(g) K_i^j and sk = sqrt(g) K.
__device__ void adm_cell_integrands(const double* __restrict__ u, long long fs, long long q,
                                   const long long st[3], double ih12, double m[3], double kk[3][3],
                                   double& sk) {
  const double W = __ldg(u + F_W * fs + q), W2 = W * W;
  double gt[6], At[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    gt[a] = __ldg(u + (F_GXX + a) * fs + q);
    At[a] = __ldg(u + (F_AXX + a) * fs + q);
  }
  // conformal inverse from the adjugate
  const double a0 = gt[3] * gt[5] - gt[4] * gt[4], a1 = gt[2] * gt[4] - gt[1] * gt[5],
               a2 = gt[1] * gt[4] - gt[2] * gt[3];
  const double det = gt[0] * a0 + gt[1] * a1 + gt[2] * a2, idet = 1.0 / det;
  const double gtu[6] = {a0 * idet, a1 * idet, a2 * idet, (gt[0] * gt[5] - gt[2] * gt[2]) * idet,
                         (gt[1] * gt[2] - gt[0] * gt[4]) * idet, (gt[0] * gt[3] - gt[1] * gt[1]) * idet};
  constexpr int S[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  // d_k g_ij = (d_k gt_ij - 2 gt_ij d_k W / W) / W^2; physical g^ij = W^2 gt^ij
  double dg[3][6];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double dWW = d1u(u + F_W * fs, q, st[d]) * ih12 / W;
#pragma unroll
    for (int a = 0; a < 6; ++a)
      dg[d][a] = (d1u(u + (F_GXX + a) * fs, q, st[d]) * ih12 - 2.0 * gt[a] * dWW) / W2;
  }
  // m^i = sqrt(g) g^ik (g^jl d_j g_kl - g^jl d_k g_jl)
  double v[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int l = 0; l < 3; ++l) s += gtu[S[j][l]] * (dg[j][S[k][l]] - dg[k][S[j][l]]);
    v[k] = W2 * s;
  }
  const double sg = sqrt(det) / (W2 * W);
#pragma unroll
  for (int i = 0; i < 3; ++i)
    m[i] = sg * W2 * (gtu[S[i][0]] * v[0] + gtu[S[i][1]] * v[1] + gtu[S[i][2]] * v[2]);
  // K_i^j = gt^jk (At_ik + gt_ik K / 3)  (the W^2 factors cancel)
  const double K = __ldg(u + F_KH * fs + q) + 2.0 * __ldg(u + F_TH * fs + q), K3 = K / 3.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double a = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) a += gtu[S[j][k]] * (At[S[i][k]] + gt[S[i][k]] * K3);
      kk[i][j] = sg * a;
    }
  sk = sg * K;
}

constexpr int ADM_THREADS = 128;
constexpr int ADM_NQ = 6;  // M, J_z, P_x, P_y, P_z, points outside

__global__ void __launch_bounds__(ADM_THREADS) adm_ring_kernel(AdmArgs A) {
  __shared__ double node[2];
  __shared__ double red[ADM_NQ][ADM_THREADS];
  const int it = blockIdx.x;
  if (threadIdx.x == 0) {
    double x, w;
    gauss_legendre_node(A.ntheta, it, x, w);
    node[0] = x;
    node[1] = w;
  }
  __syncthreads();
  const DevPatch* P = A.patches + A.patch;
  const double* __restrict__ u = P->buf[A.levels[P->level].ring];
  const long long st[3] = {1, P->px, P->plane};
  const int N[3] = {P->NX, P->NY, P->NZ};
  const double ih12 = 1.0 / (12.0 * P->dx);
  const double ct = node[0], sth = sqrt((1.0 - ct) * (1.0 + ct));
  double acc[ADM_NQ] = {0, 0, 0, 0, 0, 0};
  for (int ip = threadIdx.x; ip < A.nphi; ip += ADM_THREADS) {
    double sp, cp;
    sincospi(2.0 * ip / A.nphi, &sp, &cp);
    const double n[3] = {sth * cp, sth * sp, ct};
    double wl[3][4];
    int i0[3];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double x = A.c[d] + A.r * n[d];
      const double t = (x - P->origin[d]) / P->dx - 0.5 + GH;  // array coordinate
      ok = ok && t >= 3.0 && t < N[d] - 4.0;  // 4 interpolation cells +- 2 derivative cells inside
      i0[d] = ok ? (int)floor(t) - 1 : 0;
      cubic_weights(ok ? t - i0[d] : 0.0, wl[d]);
    }
    if (!ok) {
      acc[5] += 1.0;
      continue;
    }
    double m[3] = {0, 0, 0}, kk[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, sk = 0.0;
    for (int c = 0; c < 4; ++c)
      for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a) {
          const long long q = (i0[0] + a) + (i0[1] + b) * st[1] + (i0[2] + c) * st[2];
          double mc[3], kc[3][3], skc;
          adm_cell_integrands(u, P->fstride, q, st, ih12, mc, kc, skc);
          const double w = wl[0][a] * wl[1][b] * wl[2][c];
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            m[d] += w * mc[d];
#pragma unroll
            for (int e = 0; e < 3; ++e) kk[d][e] += w * kc[d][e];
          }
          sk += w * skc;
        }
    const double rx = A.r * n[0], ry = A.r * n[1];
    acc[0] += m[0] * n[0] + m[1] * n[1] + m[2] * n[2];
#pragma unroll
    for (int d = 0; d < 3; ++d) acc[1] += (rx * kk[1][d] - ry * kk[0][d]) * n[d];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      acc[2 + i] += kk[i][0] * n[0] + kk[i][1] * n[1] + kk[i][2] * n[2] - sk * n[i];
  }
#pragma unroll
  for (int c = 0; c < ADM_NQ; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int o = ADM_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int c = 0; c < ADM_NQ; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < ADM_NQ)
    A.ring[threadIdx.x * A.ntheta + it] = (threadIdx.x < 5 ? node[1] : 1.0) * red[threadIdx.x][0];
}

// rings in order; dS = r^2 dcos(theta) dphi with dphi = 2 pi / nphi
__global__ void adm_sum_kernel(const double* ring, int ntheta, int nphi, double r, double* out) {
  if (threadIdx.x >= ADM_NQ) return;
  const int c = threadIdx.x;
  double s = 0.0;
  for (int i = 0; i < ntheta; ++i) s += ring[c * ntheta + i];
  // (2 pi / nphi) r^2 / (16 pi) for M, / (8 pi) for J and P
  const double f = c == 0 ? r * r / (8.0 * nphi) : (c < 5 ? r * r / (4.0 * nphi) : 1.0);
  out[c] = s * f;
}

void launch_adm(const AdmArgs& a, double* out3, cudaStream_t st) {
  adm_ring_kernel<<<a.ntheta, ADM_THREADS, 0, st>>>(a);
  adm_sum_kernel<<<1, 32, 0, st>>>(a.ring, a.ntheta, a.nphi, a.r, out3);
}

}  // namespace sacrak
