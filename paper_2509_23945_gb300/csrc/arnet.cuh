// Learned slice proposal: a masked-convolution autoregressive network
// (PixelCNN masks, van den Oord et al. 2016) conditioned on the slice's field
// factors and couplings. The paper has no learned proposal; it only suggests
// replacing frequent contractions by cached knowledge of typical fields
// (Conclusions). Used as an independence proposal inside the same exact
// Metropolis-Hastings step as the tensor network (Eq. (1)).
//
// Layers l = 0..NL-1 on the active region (rows r, columns x, raster order):
//   z_l = maskconv3x3(in_l; ws_l) + conv3x3(cond; wc_l) + b_l
//   x_0 = relu(z_0); x_l = x_{l-1} + relu(z_l) for 1 <= l <= NL-2; logits = z_{NL-1}
// in_0 is the one-hot spin field with mask A (row above + left neighbour),
// in_l = x_{l-1} with mask B (mask A plus the centre). Zero padding. Taps are
// indexed t = (dy+1)*3 + (dx+1), so mask A = taps 0..3 and mask B = taps 0..4.
// Conditioning channels: log phi(v) (v < d, maximum 0, floored at -30) and
// beta*J of the right, left, lower and upper bonds of each site.
#pragma once

#include "common.cuh"
#include "fields.cuh"

namespace tnmc {

constexpr int kNetMaxLayers = 8;

struct NetLayout {
  int d, Cc, H, NL;
  int cin[kNetMaxLayers], cout[kNetMaxLayers];
  size_t off_ws[kNetMaxLayers], off_wc[kNetMaxLayers], off_b[kNetMaxLayers];
  size_t n_params;
};

inline NetLayout make_net_layout(int d, int H, int NL) {
  NetLayout n{};
  n.d = d; n.Cc = d + 4; n.H = H; n.NL = NL;
  size_t o = 0;
  for (int l = 0; l < NL; ++l) {
    n.cin[l] = l == 0 ? d : H;
    n.cout[l] = l == NL - 1 ? d : H;
    n.off_ws[l] = o; o += (size_t)n.cout[l] * n.cin[l] * 9;
    n.off_wc[l] = o; o += (size_t)n.cout[l] * n.Cc * 9;
    n.off_b[l] = o; o += (size_t)n.cout[l];
  }
  n.n_params = o;
  return n;
}

// Conditioning features of one slice into cond[c][r*Lc + x] (rows 0-based).
__device__ inline void net_cond(const Group& g, const SliceGeom& s, const int8_t* spins, const int32_t* J, double beta,
                         float* cond, int P) {
  const int d = g.d;
  const size_t vol = (size_t)g.L[0] * g.L[1] * g.L[2];
  const double b = beta * kJScale;
  for (int e = threadIdx.x; e < s.m * s.Lc; e += kThreads) {
    const int r = e / s.Lc + 1, x = e % s.Lc;
    long long h[4];
    site_field(g, s, spins, J, r, x, h);
    long long hm = h[0];
    for (int v = 1; v < d; ++v) hm = h[v] > hm ? h[v] : hm;
    for (int v = 0; v < d; ++v) {
      double lv = b * (double)(h[v] - hm);
      cond[v * P + e] = (float)(lv < -30.0 ? -30.0 : lv);
    }
    const int idx = site_index(g, s, r, x);
    const bool has_right = (x + 1 < s.Lc) || s.ring;
    const bool has_left = (x >= 1) || s.ring;
    const bool has_down = r < s.m;
    const bool has_up = r >= 2;
    double right = 0.0, left = 0.0, down = 0.0, up = 0.0;
    if (has_right) right = b * (double)J[s.ca * vol + idx];
    if (has_left) {
      const int xl = x >= 1 ? x - 1 : s.Lc - 1;
      left = b * (double)J[s.ca * vol + site_index(g, s, r, xl)];
    }
    if (has_down) down = b * (double)J[s.ra * vol + idx];
    if (has_up) up = b * (double)J[s.ra * vol + site_index(g, s, r - 1, x)];
    cond[(d + 0) * P + e] = (float)right;
    cond[(d + 1) * P + e] = (float)left;
    cond[(d + 2) * P + e] = (float)down;
    cond[(d + 3) * P + e] = (float)up;
  }
  __syncthreads();
}

__device__ inline bool tap_pos(int t, int r, int x, int m, int Lc, int* q) {
  const int rr = r + t / 3 - 1, xx = x + t % 3 - 1;
  if (rr < 0 || rr >= m || xx < 0 || xx >= Lc) return false;
  *q = rr * Lc + xx;
  return true;
}

// Teacher-forced forward of one slice. spins: [P] state indices. Stores z_l and
// x_l ([NL][H][P] each, x_{NL-1} = logits) for the backward pass.
__device__ inline void net_forward(const NetLayout& N, const float* W, const float* cond, const int8_t* spins, int m, int Lc,
                            float* zbuf, float* xbuf, int Pmax) {
  const int P = m * Lc;
  const size_t lstride = (size_t)N.H * Pmax;
  for (int l = 0; l < N.NL; ++l) {
    const int cin = N.cin[l], cout = N.cout[l];
    const int ntap = l == 0 ? 4 : 5;
    const float* ws = W + N.off_ws[l];
    const float* wc = W + N.off_wc[l];
    const float* bb = W + N.off_b[l];
    const float* xin = l > 0 ? xbuf + (size_t)(l - 1) * lstride : nullptr;
    float* z = zbuf + (size_t)l * lstride;
    float* xo = xbuf + (size_t)l * lstride;
    for (int e = threadIdx.x; e < cout * P; e += kThreads) {
      const int o = e / P, pos = e % P, r = pos / Lc, x = pos % Lc;
      float acc = bb[o];
      for (int t = 0; t < ntap; ++t) {
        int q;
        if (!tap_pos(t, r, x, m, Lc, &q)) continue;
        if (l == 0) {
          acc += ws[((size_t)o * cin + spins[q]) * 9 + t];
        } else {
          for (int i = 0; i < cin; ++i) acc += ws[((size_t)o * cin + i) * 9 + t] * xin[(size_t)i * Pmax + q];
        }
      }
      for (int t = 0; t < 9; ++t) {
        int q;
        if (!tap_pos(t, r, x, m, Lc, &q)) continue;
        for (int c = 0; c < N.Cc; ++c) acc += wc[((size_t)o * N.Cc + c) * 9 + t] * cond[(size_t)c * Pmax + q];
      }
      z[(size_t)o * Pmax + pos] = acc;
      float xv;
      if (l == N.NL - 1) xv = acc;
      else if (l == 0) xv = fmaxf(acc, 0.0f);
      else xv = xin[(size_t)o * Pmax + pos] + fmaxf(acc, 0.0f);
      xo[(size_t)o * Pmax + pos] = xv;
    }
    __syncthreads();
  }
}

// log q(s) = sum over sites of log softmax(logits)[s] (FP64 accumulation).
__device__ inline double net_logq(const NetLayout& N, const float* logits, const int8_t* spins, int P, int Pmax,
                                  double* red) {
  double loc = 0.0;
  for (int pos = threadIdx.x; pos < P; pos += kThreads) {
    double mx = -1e300;
    for (int v = 0; v < N.d; ++v) mx = fmax(mx, (double)logits[(size_t)v * Pmax + pos]);
    double se = 0.0;
    for (int v = 0; v < N.d; ++v) se += exp((double)logits[(size_t)v * Pmax + pos] - mx);
    loc += (double)logits[(size_t)spins[pos] * Pmax + pos] - mx - log(se);
  }
  return block_sum(loc, red);
}

// Raster-order draw of one slice; x_l activations are filled position by
// position (the masks make every position final once it is reached).
// condpart: [NL][H][Pmax] scratch for the conditioning stream plus bias.
__device__ inline double net_sample(const NetLayout& N, const float* W, const float* cond, int8_t* spins, int m, int Lc,
                             float* xbuf, float* condpart, int Pmax, uint64_t seed, uint32_t slice, uint32_t axis,
                             uint32_t step, uint32_t gchain, double* red, int* choice) {
  const int P = m * Lc;
  const size_t lstride = (size_t)N.H * Pmax;
  for (int l = 0; l < N.NL; ++l) {
    const float* wc = W + N.off_wc[l];
    const float* bb = W + N.off_b[l];
    float* cp = condpart + (size_t)l * lstride;
    for (int e = threadIdx.x; e < N.cout[l] * P; e += kThreads) {
      const int o = e / P, pos = e % P, r = pos / Lc, x = pos % Lc;
      float acc = bb[o];
      for (int t = 0; t < 9; ++t) {
        int q;
        if (!tap_pos(t, r, x, m, Lc, &q)) continue;
        for (int c = 0; c < N.Cc; ++c) acc += wc[((size_t)o * N.Cc + c) * 9 + t] * cond[(size_t)c * Pmax + q];
      }
      cp[(size_t)o * Pmax + pos] = acc;
    }
  }
  __syncthreads();
  double logq = 0.0;
  const int lane4 = threadIdx.x & 3;           // 4 threads per output channel
  const int og = threadIdx.x >> 2;             // 64 output groups
  for (int pos = 0; pos < P; ++pos) {
    const int r = pos / Lc, x = pos % Lc;
    for (int l = 0; l < N.NL; ++l) {
      const int cin = N.cin[l], cout = N.cout[l];
      const int ntap = l == 0 ? 4 : 5;
      const float* ws = W + N.off_ws[l];
      const float* xin = l > 0 ? xbuf + (size_t)(l - 1) * lstride : nullptr;
      float* xo = xbuf + (size_t)l * lstride;
      for (int o0 = 0; o0 < cout; o0 += kThreads / 4) {
        const int o = o0 + og;
        float acc = 0.0f;
        if (o < cout) {
          for (int t = 0; t < ntap; ++t) {
            int q;
            if (!tap_pos(t, r, x, m, Lc, &q)) continue;
            if (l == 0) {
              if (lane4 == 0) acc += ws[((size_t)o * cin + spins[q]) * 9 + t];
            } else {
              for (int i = lane4; i < cin; i += 4) acc += ws[((size_t)o * cin + i) * 9 + t] * xin[(size_t)i * Pmax + q];
            }
          }
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        if (o < cout && lane4 == 0) {
          const float zz = acc + condpart[(size_t)l * lstride + (size_t)o * Pmax + pos];
          float xv;
          if (l == N.NL - 1) xv = zz;
          else if (l == 0) xv = fmaxf(zz, 0.0f);
          else xv = xin[(size_t)o * Pmax + pos] + fmaxf(zz, 0.0f);
          xo[(size_t)o * Pmax + pos] = xv;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const float* lg = xbuf + (size_t)(N.NL - 1) * lstride;
      double mx = -1e300;
      for (int v = 0; v < N.d; ++v) mx = fmax(mx, (double)lg[(size_t)v * Pmax + pos]);
      double p[4], se = 0.0;
      for (int v = 0; v < N.d; ++v) { p[v] = exp((double)lg[(size_t)v * Pmax + pos] - mx); se += p[v]; }
      for (int v = 0; v < N.d; ++v) p[v] /= se;
      const double u = philox_uniform(seed, P_NET_SITE, (uint32_t)pos, slice, axis, step, gchain);
      double cdf = 0.0;
      int v = N.d - 1;
      for (int c = 0; c < N.d; ++c) {
        cdf += p[c];
        if (u < cdf) { v = c; break; }
      }
      spins[pos] = (int8_t)v;
      red[0] = (double)lg[(size_t)v * Pmax + pos] - mx - log(se);
    }
    __syncthreads();
    if (threadIdx.x == 0) logq += red[0];
    __syncthreads();
  }
  (void)choice;
  if (threadIdx.x == 0) red[1] = logq;
  __syncthreads();
  logq = red[1];
  __syncthreads();
  return logq;
}

// Backward of the mean NLL for one slice (weight `scale` = 1/(P * batch)),
// accumulating parameter gradients into G. gA, gB: [H][Pmax] scratch.
// g holds dL/dx_l; the relu mask is applied on the fly (gz), so the skip path
// of residual layers still sees dL/dx_l.
__device__ inline void net_backward(const NetLayout& N, const float* W, const float* cond, const int8_t* spins, int m, int Lc,
                             const float* zbuf, const float* xbuf, int Pmax, float scale, float* G, float* gA,
                             float* gB) {
  const int P = m * Lc;
  const size_t lstride = (size_t)N.H * Pmax;
  const float* lg = xbuf + (size_t)(N.NL - 1) * lstride;
  for (int pos = threadIdx.x; pos < P; pos += kThreads) {
    float mx = -1e30f;
    for (int v = 0; v < N.d; ++v) mx = fmaxf(mx, lg[(size_t)v * Pmax + pos]);
    float se = 0.0f;
    for (int v = 0; v < N.d; ++v) se += expf(lg[(size_t)v * Pmax + pos] - mx);
    for (int v = 0; v < N.d; ++v) {
      const float pv = expf(lg[(size_t)v * Pmax + pos] - mx) / se;
      gA[(size_t)v * Pmax + pos] = (pv - (spins[pos] == v ? 1.0f : 0.0f)) * scale;
    }
  }
  __syncthreads();
  float* g = gA;
  float* gn = gB;
  for (int l = N.NL - 1; l >= 0; --l) {
    const int cin = N.cin[l], cout = N.cout[l];
    const int ntap = l == 0 ? 4 : 5;
    const float* ws = W + N.off_ws[l];
    const float* z = zbuf + (size_t)l * lstride;
    const float* xin = l > 0 ? xbuf + (size_t)(l - 1) * lstride : nullptr;
    const bool last = l == N.NL - 1;
    auto gz = [&](int o, int pos) -> float {
      const float gv = g[(size_t)o * Pmax + pos];
      return (last || z[(size_t)o * Pmax + pos] > 0.0f) ? gv : 0.0f;
    };
    float* Gws = G + N.off_ws[l];
    float* Gwc = G + N.off_wc[l];
    float* Gb = G + N.off_b[l];
    for (int e = threadIdx.x; e < cout * cin * ntap; e += kThreads) {
      const int o = e / (cin * ntap), rem = e % (cin * ntap), i = rem / ntap, t = rem % ntap;
      float acc = 0.0f;
      for (int pos = 0; pos < P; ++pos) {
        int q;
        if (!tap_pos(t, pos / Lc, pos % Lc, m, Lc, &q)) continue;
        const float in = l == 0 ? (spins[q] == i ? 1.0f : 0.0f) : xin[(size_t)i * Pmax + q];
        acc += gz(o, pos) * in;
      }
      Gws[((size_t)o * cin + i) * 9 + t] += acc;
    }
    for (int e = threadIdx.x; e < cout * N.Cc * 9; e += kThreads) {
      const int o = e / (N.Cc * 9), rem = e % (N.Cc * 9), c = rem / 9, t = rem % 9;
      float acc = 0.0f;
      for (int pos = 0; pos < P; ++pos) {
        int q;
        if (!tap_pos(t, pos / Lc, pos % Lc, m, Lc, &q)) continue;
        acc += gz(o, pos) * cond[(size_t)c * Pmax + q];
      }
      Gwc[((size_t)o * N.Cc + c) * 9 + t] += acc;
    }
    for (int o = threadIdx.x; o < cout; o += kThreads) {
      float acc = 0.0f;
      for (int pos = 0; pos < P; ++pos) acc += gz(o, pos);
      Gb[o] += acc;
    }
    if (l == 0) break;
    const bool residual = l >= 1 && l <= N.NL - 2;
    // dL/dx_{l-1}: transposed masked convolution of gz, plus the skip path
    for (int e = threadIdx.x; e < cin * P; e += kThreads) {
      const int i = e / P, pos = e % P, r = pos / Lc, x = pos % Lc;
      float acc = residual ? g[(size_t)i * Pmax + pos] : 0.0f;
      for (int t = 0; t < ntap; ++t) {
        const int ro = r - (t / 3 - 1), xo = x - (t % 3 - 1);   // output that reads (r, x) through tap t
        if (ro < 0 || ro >= m || xo < 0 || xo >= Lc) continue;
        const int po = ro * Lc + xo;
        for (int o = 0; o < cout; ++o) acc += ws[((size_t)o * cin + i) * 9 + t] * gz(o, po);
      }
      gn[(size_t)i * Pmax + pos] = acc;
    }
    __syncthreads();
    float* t = g; g = gn; gn = t;
  }
  __syncthreads();
}

}  // namespace tnmc

namespace tnmc {

// Per-CTA buffers of the training / evaluation kernels (floats).
struct NetTrainParams {
  NetLayout net;
  const float* W;
  float* gbuf;            // [gridDim.x][n_params] gradient partials (each CTA owns its row)
  double* loss_part;      // [gridDim.x]
  float* ws;              // per CTA: z, x [NL][H][Pmax], gA, gB [H][Pmax], cond [Cc][Pmax], spins
  size_t ws_stride;
  int Pmax;
  // samples from the replay buffer ...
  const float* rb_cond;
  const int8_t* rb_spins;
  const int* rb_meta;
  const int* slots;       // [batch]
  int batch;
  // ... or from live slices of the lattice (evaluation hook)
  const Group* groups;
  const int* item_group;
  const int* item_chain;
  const int* item_slice;
  int axis;
  uint32_t step;
  uint64_t seed;
  float* logits_out;      // [batch][d][Pmax] (optional)
  double* logq_out;       // [batch] (optional)
  int want_grad;
};

static __global__ void __launch_bounds__(kThreads) net_train_kernel(NetTrainParams T) {
  __shared__ double red[32];
  const NetLayout& N = T.net;
  const int Pm = T.Pmax;
  float* G = T.gbuf ? T.gbuf + (size_t)blockIdx.x * N.n_params : nullptr;
  if (G)
    for (size_t p = threadIdx.x; p < N.n_params; p += kThreads) G[p] = 0.0f;
  float* zb = T.ws + (size_t)blockIdx.x * T.ws_stride;
  float* xb = zb + (size_t)N.NL * N.H * Pm;
  float* gA = xb + (size_t)N.NL * N.H * Pm;
  float* gB = gA + (size_t)N.H * Pm;
  float* condb = gB + (size_t)N.H * Pm;
  int8_t* sb = reinterpret_cast<int8_t*>(condb + (size_t)N.Cc * Pm);
  __syncthreads();
  double loss = 0.0;
  for (int b = blockIdx.x; b < T.batch; b += gridDim.x) {
    const float* cond;
    const int8_t* spins;
    int m, Lc;
    if (T.slots) {
      const int slot = T.slots[b];
      m = T.rb_meta[2 * slot];
      Lc = T.rb_meta[2 * slot + 1];
      cond = T.rb_cond + (size_t)slot * N.Cc * Pm;
      spins = T.rb_spins + (size_t)slot * Pm;
    } else {
      const Group& g = T.groups[T.item_group[b]];
      const int chain = T.item_chain[b];
      const uint32_t gchain = (uint32_t)(g.chain_base + chain);
      const SliceGeom s = make_geom(g, T.axis, T.item_slice[b], T.seed, T.step, gchain);
      const size_t vol = (size_t)g.L[0] * g.L[1] * g.L[2];
      const int8_t* lat = g.spins + (size_t)chain * vol;
      const int32_t* J = g.J + (size_t)g.inst[chain] * 3 * vol;
      net_cond(g, s, lat, J, g.beta[chain], condb, Pm);
      for (int e = threadIdx.x; e < s.m * s.Lc; e += kThreads) sb[e] = lat[site_index(g, s, e / s.Lc + 1, e % s.Lc)];
      __syncthreads();
      m = s.m;
      Lc = s.Lc;
      cond = condb;
      spins = sb;
    }
    const int P = m * Lc;
    net_forward(N, T.W, cond, spins, m, Lc, zb, xb, Pm);
    const float* lg = xb + (size_t)(N.NL - 1) * N.H * Pm;
    const double lq = net_logq(N, lg, spins, P, Pm, red);
    loss += -lq / (double)P;
    if (T.logq_out && threadIdx.x == 0) T.logq_out[b] = lq;
    if (T.logits_out)
      for (int e = threadIdx.x; e < N.d * Pm; e += kThreads)
        T.logits_out[(size_t)b * N.d * Pm + e] = (e % Pm) < P ? lg[e] : 0.0f;
    if (T.want_grad) net_backward(N, T.W, cond, spins, m, Lc, zb, xb, Pm, 1.0f / ((float)P * T.batch), G, gA, gB);
    __syncthreads();
  }
  if (threadIdx.x == 0 && T.loss_part) T.loss_part[blockIdx.x] = loss;
}

// Sum the per-CTA gradient rows in a fixed order, optionally export the sum,
// and apply one Adam step (Kingma & Ba 2015, bias-corrected) when lr > 0.
static __global__ void net_adam_kernel(size_t n, float* W, float* m1, float* m2, const float* gbuf, int rows, float lr,
                                float b1, float b2, float eps, int t, float* gout) {
  const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    float g = 0.0f;
    for (int r = 0; r < rows; ++r) g += gbuf[(size_t)r * n + p];
    if (gout) gout[p] = g;
    if (lr > 0.0f) {
      const float a = b1 * m1[p] + (1.0f - b1) * g;
      const float b = b2 * m2[p] + (1.0f - b2) * g * g;
      m1[p] = a;
      m2[p] = b;
      W[p] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    }
  }
}

// He-style uniform initialisation from Philox draws: w ~ U(-a, a), a = sqrt(6 / fan_in),
// the output layer scaled by 0.1 and biases zero.
static __global__ void net_init_kernel(NetLayout N, float* W, uint64_t seed) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N.n_params; p += (size_t)gridDim.x * blockDim.x) {
    int l = 0;
    while (l + 1 < N.NL && p >= N.off_ws[l + 1]) ++l;
    float val = 0.0f;
    if (p < N.off_b[l]) {
      const float fan = (float)(N.cin[l] * 9 + N.Cc * 9);
      const double u = philox_uniform(seed, 7u, (uint32_t)(p & 0xffffff), (uint32_t)(p >> 24), 0, 0, 0);
      val = (float)(2.0 * u - 1.0) * sqrtf(6.0f / fan) * (l == N.NL - 1 ? 0.1f : 1.0f);
    }
    W[p] = val;
  }
}

}  // namespace tnmc
