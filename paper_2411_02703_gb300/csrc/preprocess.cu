// preprocess.cu -- per-Gaussian projection (a1) and its chain rule (a7).
//
// Forward, one warp per 32 Gaussians (the pairs in front of the near plane
// dealt out over the lanes), for every view of the call:
//   Sigma = R S S^T R^T (Eq. 2), the EWA projection Sigma_I = J Q Sigma Q^T J^T
//   and mu_I = [Q, T] mu (Eq. 7), the 0.3 px^2 dilation, the conic, the 3-sigma
//   radius and tile rectangle, opacity = sigmoid(logit) and the SH colour.
// The quantities that decide the tile keys (view-space z, screen position,
// radius, rectangle) are evaluated in strict IEEE binary32 with one rounding
// per operation in a fixed order (the __f*_rn intrinsics are never
// contracted), so the keys are reproducible bit for bit on any IEEE machine.
//
// Backward, one warp per 32 Gaussians: the visible (view, Gaussian) pairs are
// dealt out over the lanes and summed per Gaussian in shared memory (plain
// adds, the lanes of one owner taking turns), so the parameter gradients need
// no atomics.
#include <cmath>

#include "lvigs_internal.cuh"

namespace lvigs {
namespace {

#define RN_MUL __fmul_rn
#define RN_ADD __fadd_rn
#define RN_SUB __fsub_rn
#define RN_DIV __fdiv_rn

// Real spherical-harmonic normalisations (with the Condon-Shortley phase).
constexpr float kY00 = 0.28209479177387814f;  // 1 / (2 sqrt(pi))
constexpr float kY1 = 0.48860251190291992f;   // sqrt(3 / (4 pi))
constexpr float kY2a = 1.0925484305920792f;   // sqrt(15 / pi) / 2
constexpr float kY2b = 0.31539156525252005f;  // sqrt(5 / pi) / 4
constexpr float kY2c = 0.54627421529603959f;  // sqrt(15 / pi) / 4
constexpr float kY3a = 0.59004358992664352f;  // sqrt(35 / (2 pi)) / 4
constexpr float kY3b = 2.8906114426405538f;   // sqrt(105 / pi) / 2
constexpr float kY3c = 0.45704579946446572f;  // sqrt(21 / (2 pi)) / 4
constexpr float kY3d = 0.37317633259011540f;  // sqrt(7 / pi) / 4
constexpr float kY3e = 1.4453057213202769f;   // sqrt(105 / pi) / 4

// Basis values at the unit direction (x, y, z), index l^2 + l + m.
__device__ __forceinline__ void sh_values(int deg, float x, float y, float z, float Y[16]) {
    Y[0] = kY00;
    if (deg < 1) return;
    Y[1] = -kY1 * y;
    Y[2] = kY1 * z;
    Y[3] = -kY1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kY2a * x * y;
    Y[5] = -kY2a * y * z;
    Y[6] = kY2b * (2.f * zz - xx - yy);
    Y[7] = -kY2a * x * z;
    Y[8] = kY2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = -kY3a * y * (3.f * xx - yy);
    Y[10] = kY3b * x * y * z;
    Y[11] = -kY3c * y * (4.f * zz - xx - yy);
    Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -kY3c * x * (4.f * zz - xx - yy);
    Y[14] = kY3e * z * (xx - yy);
    Y[15] = -kY3a * x * (xx - 3.f * yy);
}

// sum_k w[k] * grad Y_k at (x, y, z), with the Cartesian gradient of each
// basis polynomial (the projection onto the sphere is applied by the caller).
__device__ __forceinline__ float3 sh_weighted_grad(int deg, float x, float y, float z,
                                                   const float w[16]) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (deg >= 1) {
        gy -= kY1 * w[1];
        gz += kY1 * w[2];
        gx -= kY1 * w[3];
    }
    if (deg >= 2) {
        gx += kY2a * y * w[4];
        gy += kY2a * x * w[4];
        gy -= kY2a * z * w[5];
        gz -= kY2a * y * w[5];
        gx -= 2.f * kY2b * x * w[6];
        gy -= 2.f * kY2b * y * w[6];
        gz += 4.f * kY2b * z * w[6];
        gx -= kY2a * z * w[7];
        gz -= kY2a * x * w[7];
        gx += 2.f * kY2c * x * w[8];
        gy -= 2.f * kY2c * y * w[8];
    }
    if (deg >= 3) {
        const float xx = x * x, yy = y * y, zz = z * z;
        gx -= 6.f * kY3a * x * y * w[9];
        gy -= 3.f * kY3a * (xx - yy) * w[9];
        gx += kY3b * y * z * w[10];
        gy += kY3b * x * z * w[10];
        gz += kY3b * x * y * w[10];
        gx += 2.f * kY3c * x * y * w[11];
        gy -= kY3c * (4.f * zz - xx - 3.f * yy) * w[11];
        gz -= 8.f * kY3c * y * z * w[11];
        gx -= 6.f * kY3d * x * z * w[12];
        gy -= 6.f * kY3d * y * z * w[12];
        gz += kY3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
        gx -= kY3c * (4.f * zz - 3.f * xx - yy) * w[13];
        gy += 2.f * kY3c * x * y * w[13];
        gz -= 8.f * kY3c * x * z * w[13];
        gx += 2.f * kY3e * x * z * w[14];
        gy -= 2.f * kY3e * y * z * w[14];
        gz += kY3e * (xx - yy) * w[14];
        gx -= 3.f * kY3a * (xx - yy) * w[15];
        gy += 6.f * kY3a * x * y * w[15];
    }
    return make_float3(gx, gy, gz);
}

// Rotation of the unit quaternion (w, x, y, z), strict binary32.
__device__ __forceinline__ void quat_rotation_strict(float w, float x, float y, float z, float r[9]) {
    r[0] = RN_SUB(1.f, RN_MUL(2.f, RN_ADD(RN_MUL(y, y), RN_MUL(z, z))));
    r[1] = RN_MUL(2.f, RN_SUB(RN_MUL(x, y), RN_MUL(w, z)));
    r[2] = RN_MUL(2.f, RN_ADD(RN_MUL(x, z), RN_MUL(w, y)));
    r[3] = RN_MUL(2.f, RN_ADD(RN_MUL(x, y), RN_MUL(w, z)));
    r[4] = RN_SUB(1.f, RN_MUL(2.f, RN_ADD(RN_MUL(x, x), RN_MUL(z, z))));
    r[5] = RN_MUL(2.f, RN_SUB(RN_MUL(y, z), RN_MUL(w, x)));
    r[6] = RN_MUL(2.f, RN_SUB(RN_MUL(x, z), RN_MUL(w, y)));
    r[7] = RN_MUL(2.f, RN_ADD(RN_MUL(y, z), RN_MUL(w, x)));
    r[8] = RN_SUB(1.f, RN_MUL(2.f, RN_ADD(RN_MUL(x, x), RN_MUL(y, y))));
}

__device__ __forceinline__ float dot3_strict(float a0, float a1, float a2, float b0, float b1,
                                             float b2) {
    return RN_ADD(RN_ADD(RN_MUL(a0, b0), RN_MUL(a1, b1)), RN_MUL(a2, b2));
}

__device__ __forceinline__ float tile_coord(float f, int hi) {
    if (!(f > 0.f)) return 0.f;
    if (f > (float)hi) return (float)hi;
    return f;
}

// exp(x) rounded once to binary32, the value (float)exp((double)x) of the key
// stage, without binary64 arithmetic on the common path (binary64 runs at a
// small fraction of the binary32 rate on this GPU).  Tang's table-driven
// reduction: x = (32 m + j) ln2/32 + r, |r| <= ln2/64, with ln2/32 split in
// three parts (the first two of 12 significant bits, so k times each is exact)
// and r kept as a normalised float pair; exp(r) - 1 = r + r^2/2 + r^3/6 + r^4/24 (the
// truncation is below 2^-39); 2^(j/32) is a float pair from the table; the
// products and sums that matter are exact (FMA products, two-sums).  The
// result y = z + d (z the nearest float) is within about 2^-36 relative of
// exp(x); when the rounding of z is not certain by a margin of 1e-10 z (the
// exact value may lie across a rounding boundary), or |x| >= 60, the binary64
// path decides.  So the result is always the binary64 path's.
__device__ __forceinline__ float exp_key(float x, const ExpKeyTable &t) {
    if (!(fabsf(x) < 60.f)) return __double2float_rn(exp((double)x));
    // (explicitly rounded operations: none of the exact steps may be contracted)
    const float kf = rintf(RN_MUL(x, t.inv_step));
    const int k = (int)kf;
    const int j = k & 31, m = k >> 5;
    // r = x - k ln2/32 = rh + rl
    const float r1 = __fmaf_rn(-kf, t.c1, x); // exact
    const float p2 = RN_MUL(kf, t.c2);         // exact
    const float r2 = RN_SUB(r1, p2);
    const float bv = RN_SUB(r2, r1);
    const float er = RN_ADD(RN_SUB(r1, RN_SUB(r2, bv)), RN_SUB(-p2, bv)); // two-sum error
    const float r3 = __fmaf_rn(-kf, t.c3, er); // up to about 1e-6: renormalise the pair
    const float rh = RN_ADD(r2, r3);
    const float bu = RN_SUB(rh, r2);
    const float rl = RN_ADD(RN_SUB(r2, RN_SUB(rh, bu)), RN_SUB(r3, bu));
    const float q = RN_MUL(RN_MUL(rh, rh), __fmaf_rn(rh, __fmaf_rn(rh, 1.f / 24.f, 1.f / 6.f), 0.5f));
    const float pl = RN_ADD(rl, q); // exp(r) = 1 + rh + pl
    // y = 2^(j/32) (1 + rh + pl), 2^(j/32) = th + tl
    const float th = t.hi[j], tl = t.lo[j];
    const float pr = RN_MUL(th, rh);
    const float pe = __fmaf_rn(th, rh, -pr); // exact product error
    const float yh = RN_ADD(th, pr);
    const float bw = RN_SUB(yh, th);
    const float e2 = RN_ADD(RN_SUB(th, RN_SUB(yh, bw)), RN_SUB(pr, bw));
    // the rest of (th + tl)(1 + rh + pl): th pl + tl (1 + rh) (tl pl is below 2^-39)
    const float yl = RN_ADD(RN_ADD(e2, pe), __fmaf_rn(th, pl, __fmaf_rn(tl, rh, tl)));
    const float z = RN_ADD(yh, yl);
    const float d = RN_ADD(RN_SUB(yh, z), yl);
    const uint32_t zb = __float_as_uint(z);
    const float u = RN_SUB(__uint_as_float(zb + 1u), z);
    const bool pow2 = (zb & 0x7fffffu) == 0u;
    const float room = d >= 0.f ? RN_SUB(RN_MUL(0.5f, u), d) : RN_ADD(RN_MUL(pow2 ? 0.25f : 0.5f, u), d);
    if (!(room > RN_MUL(1e-10f, z))) return __double2float_rn(exp((double)x));
    return ldexpf(z, m);
}

// Per-Gaussian, view-independent part: scales, unit quaternion, Sigma (strict).
struct GaussLocal {
    float s[3];
    float qn[4];
    float qnorm;
    float r[9];
    float S[6]; // Sigma00, 01, 02, 11, 12, 22
    bool ok;
};

__device__ __forceinline__ void gauss_local_strict(const GaussParams &P, int g, GaussLocal &L,
                                                   const ExpKeyTable &et) {
    const float *ls = P.log_scales + 3 * (size_t)g;
    const float *q = P.quats + 4 * (size_t)g;
    // exp as in binary64, one rounding to binary32
    L.s[0] = exp_key(ls[0], et);
    L.s[1] = exp_key(ls[1], et);
    L.s[2] = exp_key(ls[2], et);
    const float q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
    float n2 = RN_MUL(q0, q0);
    n2 = RN_ADD(n2, RN_MUL(q1, q1));
    n2 = RN_ADD(n2, RN_MUL(q2, q2));
    n2 = RN_ADD(n2, RN_MUL(q3, q3));
    L.ok = n2 > 0.f;
    const float nr = __fsqrt_rn(n2);
    L.qnorm = nr;
    L.qn[0] = RN_DIV(q0, nr);
    L.qn[1] = RN_DIV(q1, nr);
    L.qn[2] = RN_DIV(q2, nr);
    L.qn[3] = RN_DIV(q3, nr);
    quat_rotation_strict(L.qn[0], L.qn[1], L.qn[2], L.qn[3], L.r);
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) M[3 * i + j] = RN_MUL(L.r[3 * i + j], L.s[j]);
    L.S[0] = dot3_strict(M[0], M[1], M[2], M[0], M[1], M[2]);
    L.S[1] = dot3_strict(M[0], M[1], M[2], M[3], M[4], M[5]);
    L.S[2] = dot3_strict(M[0], M[1], M[2], M[6], M[7], M[8]);
    L.S[3] = dot3_strict(M[3], M[4], M[5], M[3], M[4], M[5]);
    L.S[4] = dot3_strict(M[3], M[4], M[5], M[6], M[7], M[8]);
    L.S[5] = dot3_strict(M[6], M[7], M[8], M[6], M[7], M[8]);
}

__device__ __forceinline__ float sig(const float S[6], int i, int j) {
    // symmetric access into the 6 stored entries
    const int lo = i < j ? i : j, hi = i < j ? j : i;
    return S[lo == 0 ? hi : (lo == 1 ? 2 + hi : 5)];
}

constexpr int kShRow = 48;   // 16 coefficients x 3 channels
constexpr int kShPitch = 49; // staged row pitch: odd, so lanes reading 32 rows hit 32 banks

// A warp's 32 consecutive SH rows (one contiguous run of nrows * row floats)
// into dst at pitch kShPitch: float4 loads all issued before the stores when
// the run is 16-byte aligned.  ROW is the row length when known at compile
// time (the degree-3 row; the element's row then comes from a constant
// divide), else 0 and `row` gives it.  row <= kShRow.
template <int ROW>
__device__ __forceinline__ void stage_sh_rows_t(const float *__restrict__ src, int nrows, int row, int lane,
                                                float *__restrict__ dst) {
    if (ROW) row = ROW;
    const int n = nrows * row;
    // (only the compile-time row takes the unrolled path: one copy of it keeps
    // the kernels' code small)
    if (ROW && (((uintptr_t)src) & 15u) == 0 && (n & 3) == 0) {
        constexpr int kMaxIt = 32 * kShRow / 4 / 32;
        float4 v[kMaxIt];
#pragma unroll
        for (int i = 0; i < kMaxIt; ++i) {
            const int e4 = lane + 32 * i;
            if (4 * e4 < n) v[i] = __ldg(reinterpret_cast<const float4 *>(src) + e4);
        }
#pragma unroll
        for (int i = 0; i < kMaxIt; ++i) {
            const int e = 4 * (lane + 32 * i);
            if (e < n) {
                const float f[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int rr = (e + c) / row, cc = (e + c) - rr * row;
                    dst[rr * kShPitch + cc] = f[c];
                }
            }
        }
    } else {
        for (int e = lane; e < n; e += 32) {
            const int rr = e / row, cc = e - rr * row;
            dst[rr * kShPitch + cc] = __ldg(src + e);
        }
    }
}

__device__ __forceinline__ void stage_sh_rows(const float *__restrict__ src, int nrows, int row, int lane,
                                              float *__restrict__ dst) {
    if (row == kShRow) stage_sh_rows_t<kShRow>(src, nrows, row, lane, dst);
    else stage_sh_rows_t<0>(src, nrows, row, lane, dst);
}

// mu_I = [Q_iw, T_iw] mu_W (Eq. 7), strict binary32.
__device__ __forceinline__ void view_point_strict(const ViewDesc &V, float mx, float my, float mz, float &px,
                                                  float &py, float &pz) {
    px = RN_MUL(V.R[0], mx);
    px = RN_ADD(px, RN_MUL(V.R[1], my));
    px = RN_ADD(px, RN_MUL(V.R[2], mz));
    px = RN_ADD(px, V.t[0]);
    py = RN_MUL(V.R[3], mx);
    py = RN_ADD(py, RN_MUL(V.R[4], my));
    py = RN_ADD(py, RN_MUL(V.R[5], mz));
    py = RN_ADD(py, V.t[1]);
    pz = RN_MUL(V.R[6], mx);
    pz = RN_ADD(pz, RN_MUL(V.R[7], my));
    pz = RN_ADD(pz, RN_MUL(V.R[8], mz));
    pz = RN_ADD(pz, V.t[2]);
}

// Forward (a1).  A warp owns 32 consecutive Gaussians.  Every lane first
// projects its Gaussian's mean into every view (depth key bits for all pairs);
// the pairs in front of the near plane are then dealt out over all 32 lanes
// for the projected covariance, radius, tile rectangle, SH colour and record,
// the worker taking the owner's mean, Sigma and opacity by shuffle and its SH
// row from shared memory (staged with coalesced loads).
constexpr int kFwdThreads = 128;

__global__ void __launch_bounds__(kFwdThreads)
preprocess_fwd_kernel(GaussParams P, const ViewSet *__restrict__ vsp, GRec *__restrict__ recs,
                      uint32_t *__restrict__ tiles, uint32_t *__restrict__ zbits,
                      uint2 *__restrict__ rects, GGrad *__restrict__ g2d_init, ExpKeyTable et_param) {
    __shared__ float s_sh[kFwdThreads / 32][32 * kShPitch];
    __shared__ ExpKeyTable et;
    if (threadIdx.x < 32) {
        et.hi[threadIdx.x] = et_param.hi[threadIdx.x];
        et.lo[threadIdx.x] = et_param.lo[threadIdx.x];
    }
    if (threadIdx.x == 0) {
        et.inv_step = et_param.inv_step;
        et.c1 = et_param.c1;
        et.c2 = et_param.c2;
        et.c3 = et_param.c3;
    }
    __syncthreads();
    __shared__ uint32_t s_mask[kFwdThreads / 32][kMaxViews];
    __shared__ int s_pref[kFwdThreads / 32][kMaxViews + 1];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t N = P.n;
    const int64_t g0 = (int64_t)blockIdx.x * kFwdThreads + (tid & ~31);
    const int64_t g = g0 + lane;
    const bool valid = g < N;
    const int nrows = (int)(N - g0 < 32 ? N - g0 : 32);
    if (nrows <= 0) return; // whole warp past the end (warp-uniform)
    const int deg = P.sh_degree;
    const int nk = (deg + 1) * (deg + 1);
    const int row = P.sh_stride_k * 3;
    const bool staged = row <= kShRow;
    if (staged) stage_sh_rows(P.sh + g0 * row, nrows, row, lane, s_sh[w]);

    GaussLocal L;
    L.ok = false;
#pragma unroll
    for (int i = 0; i < 6; ++i) L.S[i] = 0.f;
    float mx = 0.f, my = 0.f, mz = 0.f, opacity = 0.f;
    if (valid) {
        gauss_local_strict(P, (int)g, L, et);
        mx = P.means[3 * g];
        my = P.means[3 * g + 1];
        mz = P.means[3 * g + 2];
        opacity = 1.f / (1.f + expf(-P.opacity_logits[g]));
    }
    const float tw = (float)vsp->tile_w, th = (float)vsp->tile_h;
    // tile sizes are powers of two (8, 16, 32): the reciprocals are exact and
    // a product with one is the correctly rounded quotient, bit for bit
    const float itw = 1.f / tw, ith = 1.f / th;
    const int n_views = vsp->n_views;

    // depth key of every pair; pairs in front of the near plane go on to the rest
    for (int vi = 0; vi < n_views; ++vi) {
        bool front = false;
        if (valid) {
            const size_t o = (size_t)vi * N + g;
            float px, py, pz;
            view_point_strict(vsp->v[vi], mx, my, mz, px, py, pz);
            front = L.ok && (pz > 0.2f);
            zbits[o] = __float_as_uint(pz);
            if (!front) tiles[o] = 0; // (its rectangle is never read)
        }
        const uint32_t m = __ballot_sync(0xffffffffu, front);
        if (lane == 0) s_mask[w][vi] = m;
    }
    __syncwarp();
    if (lane == 0) {
        int acc = 0;
        for (int vi = 0; vi < n_views; ++vi) {
            s_pref[w][vi] = acc;
            acc += __popc(s_mask[w][vi]);
        }
        s_pref[w][n_views] = acc;
    }
    __syncwarp();
    const int total = s_pref[w][n_views];

    for (int base = 0; base < total; base += 32) {
        const int p = base + lane;
        const bool has = p < total;
        int vi = 0, src = lane;
        if (has) {
            while (vi + 1 < n_views && s_pref[w][vi + 1] <= p) ++vi;
            src = (int)__fns(s_mask[w][vi], 0, p - s_pref[w][vi] + 1);
        }
        const float gx = __shfl_sync(0xffffffffu, mx, src);
        const float gy = __shfl_sync(0xffffffffu, my, src);
        const float gz = __shfl_sync(0xffffffffu, mz, src);
        const float op = __shfl_sync(0xffffffffu, opacity, src);
        float S[6];
#pragma unroll
        for (int t = 0; t < 6; ++t) S[t] = __shfl_sync(0xffffffffu, L.S[t], src);
        if (!has) continue;
        const ViewDesc &V = vsp->v[vi];
        const size_t o = (size_t)vi * N + (size_t)(g0 + src);
        float px, py, pz;
        view_point_strict(V, gx, gy, gz, px, py, pz);
        bool vis = true;
        float a = 0.f, b = 0.f, c = 0.f, det = 0.f, u = 0.f, v = 0.f;
        int rad = 0;
        {
            const float xz = RN_DIV(px, pz), yz = RN_DIV(py, pz);
            const float txc = xz < -V.limx ? -V.limx : (xz > V.limx ? V.limx : xz);
            const float tyc = yz < -V.limy ? -V.limy : (yz > V.limy ? V.limy : yz);
            const float J00 = RN_DIV(V.fx, pz);
            const float J02 = RN_DIV(-RN_MUL(V.fx, txc), pz);
            const float J11 = RN_DIV(V.fy, pz);
            const float J12 = RN_DIV(-RN_MUL(V.fy, tyc), pz);
            float T[6];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T[j] = RN_ADD(RN_MUL(J00, V.R[j]), RN_MUL(J02, V.R[6 + j]));
                T[3 + j] = RN_ADD(RN_MUL(J11, V.R[3 + j]), RN_MUL(J12, V.R[6 + j]));
            }
            float U[6];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float acc = RN_MUL(T[3 * i], sig(S, 0, j));
                    acc = RN_ADD(acc, RN_MUL(T[3 * i + 1], sig(S, 1, j)));
                    acc = RN_ADD(acc, RN_MUL(T[3 * i + 2], sig(S, 2, j)));
                    U[3 * i + j] = acc;
                }
            a = dot3_strict(U[0], U[1], U[2], T[0], T[1], T[2]);
            b = dot3_strict(U[0], U[1], U[2], T[3], T[4], T[5]);
            c = dot3_strict(U[3], U[4], U[5], T[3], T[4], T[5]);
            a = RN_ADD(a, 0.3f);
            c = RN_ADD(c, 0.3f);
            det = RN_SUB(RN_MUL(a, c), RN_MUL(b, b));
            vis = det > 0.f;
            if (vis) {
                const float mid = RN_MUL(0.5f, RN_ADD(a, c));
                const float disc = RN_SUB(RN_MUL(mid, mid), det);
                const float lam = RN_ADD(mid, __fsqrt_rn(disc > 0.1f ? disc : 0.1f));
                rad = (int)ceilf(RN_MUL(3.f, __fsqrt_rn(lam)));
                u = RN_ADD(RN_MUL(V.fx, xz), V.cx);
                v = RN_ADD(RN_MUL(V.fy, yz), V.cy);
            }
        }
        uint32_t ntiles = 0;
        uint2 rect = make_uint2(0, 0);
        if (vis) {
            const float fr = (float)rad;
            const int x0 = (int)tile_coord(RN_MUL(RN_SUB(u, fr), itw), V.tiles_x);
            const int x1 = (int)tile_coord(RN_MUL(RN_ADD(RN_ADD(u, fr), tw - 1.f), itw), V.tiles_x);
            const int y0 = (int)tile_coord(RN_MUL(RN_SUB(v, fr), ith), V.tiles_y);
            const int y1 = (int)tile_coord(RN_MUL(RN_ADD(RN_ADD(v, fr), th - 1.f), ith), V.tiles_y);
            ntiles = (uint32_t)((x1 - x0) * (y1 - y0));
            rect = make_uint2((uint32_t)x0 | ((uint32_t)x1 << 16), (uint32_t)y0 | ((uint32_t)y1 << 16));
        }
        tiles[o] = ntiles;
        rects[o] = rect;
        if (ntiles == 0) continue;
        // values composited (binary32; not part of the key)
        const float inv_det = 1.f / det;
        // colour: SH at the direction from the camera centre to the mean
        float dx = gx - V.campos[0], dy = gy - V.campos[1], dz = gz - V.campos[2];
        const float inv_len = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= inv_len;
        dy *= inv_len;
        dz *= inv_len;
        float Y[16];
        sh_values(deg, dx, dy, dz, Y);
        const float *shg = staged ? &s_sh[w][src * kShPitch] : P.sh + (size_t)(g0 + src) * row;
        float rgb[3];
        uint32_t clamp = kClampKnown;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.5f;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if (k < nk) acc += Y[k] * shg[3 * k + ch];
            if (acc < 0.f) clamp |= 1u << ch;
            rgb[ch] = fmaxf(acc, 0.f);
        }
        if (g2d_init) {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            g2d_init[o] = GGrad{z, z, make_float4(0.f, 0.f, 0.f, __uint_as_float(clamp))};
        }
        // half-extents of the box where o exp(power) can reach 1/255: the
        // ellipse d^T Sigma_I^{-1} d <= 2 (ln(255 o) + 0.1), widened by 0.05 px;
        // the margin is far above the binary32 rounding of the compositing test
        float ex = -1e30f, ey = -1e30f;
        if (op * 255.f >= 1.f) {
            const float tau = logf(255.f * op) + 0.1f;
            ex = (a > 0.f) ? sqrtf(2.f * tau * a) + 0.05f : 1e30f;
            ey = (c > 0.f) ? sqrtf(2.f * tau * c) + 0.05f : 1e30f;
        }
        // conic [[A, B], [B, C]] = [[c, -b], [-b, a]] / det, stored as the
        // coefficients of the base-2 exponent log2(e) * power (see GRec)
        constexpr float kLog2e = 1.4426950408889634f;
        GRec rec;
        rec.a = make_float4(u, v, (c * inv_det) * (-0.5f * kLog2e), (b * inv_det) * kLog2e);
        rec.b = make_float4((a * inv_det) * (-0.5f * kLog2e), log2f(op), pz, ex);
        rec.c = make_float4(rgb[0], rgb[1], rgb[2], ey);
        recs[o] = rec;
    }
}

// ---------------------------------------------------------------------------
// Backward (a7): chain rule from the screen-space gradients of every view.
//
// A warp owns 32 consecutive Gaussians.  Their visible (view, Gaussian) pairs
// (on average a third of the views) are enumerated warp-wide and dealt out to
// all 32 lanes, so the per-view chain rule runs with full lanes instead of one
// lane per Gaussian idling through the views it does not see.  The worker lane
// takes the owner's mean and Sigma by shuffle and its SH row from shared
// memory (staged with coalesced loads), and adds its terms to the owner's
// accumulators in shared memory.  A round of 32 pairs spans a few views, so
// an owner can appear in several lanes of it: those lanes add in lane order,
// one turn each (match_any ranks them), which keeps the adds plain (a
// shared-memory float atomic costs far more) and the sums deterministic.  The owner then finishes the per-Gaussian
// part (Sigma -> scale, rotation; opacity) and the warp writes the SH
// gradient rows back coalesced.
// ---------------------------------------------------------------------------
constexpr int kBwdThreads = 128;
constexpr int kAccScalars = 10; // d_mean 3, dSigma 6 (00,01,02,11,12,22), d_opacity 1
constexpr size_t kBwdSmem = sizeof(float) * ((kAccScalars + kShRow) * (kBwdThreads + 1) + kBwdThreads * kShPitch) +
                            sizeof(uint32_t) * (kBwdThreads / 32) * kMaxViews +
                            sizeof(int) * (kBwdThreads / 32) * (kMaxViews + 1);

// Rows [0, nrows) of the warp's SH gradients from the accumulators (column
// wbase + row, one accumulator row per coefficient-channel at pitch ld) to
// dst, consecutive lanes on consecutive floats; columns from `live` on are
// zero (left as they are when accumulating).  ROW as in stage_sh_rows_t; with
// ROW and a 16-byte aligned dst the run moves as float4, and when
// accumulating every load of a lane is issued before its first store.
template <int ROW>
__device__ __forceinline__ void write_sh_grad_rows(float *__restrict__ dst, int nrows, int row, int live_cols,
                                                   const float *__restrict__ acc, int ld, int wbase, int lane,
                                                   int accumulate) {
    if (ROW) row = ROW;
    const int n = nrows * row;
    if (ROW && (ROW & 3) == 0 && (((uintptr_t)dst) & 15u) == 0) {
        constexpr int kIt = 32 * (ROW ? ROW : 4) / 4 / 32;
        float4 old[kIt];
        if (accumulate) {
#pragma unroll
            for (int i = 0; i < kIt; ++i) {
                const int e4 = lane + 32 * i;
                if (4 * e4 < n) old[i] = reinterpret_cast<const float4 *>(dst)[e4];
            }
        }
#pragma unroll
        for (int i = 0; i < kIt; ++i) {
            const int e = 4 * (lane + 32 * i);
            if (e >= n) continue;
            float v[4], o[4] = {0.f, 0.f, 0.f, 0.f};
            if (accumulate) {
                o[0] = old[i].x;
                o[1] = old[i].y;
                o[2] = old[i].z;
                o[3] = old[i].w;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                constexpr int R = ROW ? ROW : 1; // (this branch is taken with ROW only)
                const int rw = (e + c) / R, col = (e + c) - rw * R;
                const bool live = col < live_cols && col < kShRow;
                v[c] = live ? (accumulate ? o[c] + acc[col * ld + wbase + rw] : acc[col * ld + wbase + rw])
                            : (accumulate ? o[c] : 0.f);
            }
            reinterpret_cast<float4 *>(dst)[e / 4] = make_float4(v[0], v[1], v[2], v[3]);
        }
        return;
    }
    for (int e = lane; e < n; e += 32) {
        const int rw = e / row, col = e - rw * row;
        const bool live = col < live_cols && col < kShRow;
        const float v = live ? acc[col * ld + wbase + rw] : 0.f;
        if (!accumulate) dst[e] = v;
        else if (live) dst[e] += v;
    }
}

__global__ void __launch_bounds__(kBwdThreads, 4)
preprocess_bwd_kernel(GaussParams P, const ViewSet *__restrict__ vsp, const uint32_t *__restrict__ tiles,
                      const GGrad *__restrict__ g2d, ParamGrads G) {
    // accumulators [quantity][owner thread] (+1 column: conflict-free transposed
    // reads), the warps' SH rows, per-view visibility masks and their prefix counts
    extern __shared__ float4 smem_bwd[];
    auto s_sh = reinterpret_cast<float(*)[32 * kShPitch]>(smem_bwd);
    auto s_acc = reinterpret_cast<float(*)[kBwdThreads + 1]>(&s_sh[kBwdThreads / 32][0]);
    auto s_mask = reinterpret_cast<uint32_t(*)[kMaxViews]>(&s_acc[kAccScalars + kShRow][0]);
    auto s_pref = reinterpret_cast<int(*)[kMaxViews + 1]>(&s_mask[kBwdThreads / 32][0]);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, wbase = tid & ~31;
    const int64_t N = P.n;
    const int64_t g0 = (int64_t)blockIdx.x * kBwdThreads + wbase; // first Gaussian of the warp
    const int64_t g = g0 + lane;
    const bool valid = g < N;
    const int deg = P.sh_degree;
    const int nk = (deg + 1) * (deg + 1);
    const int K = P.sh_stride_k;
    const int row = K * 3;
    const bool staged = row <= kShRow;
    const int nrows = (int)(N - g0 < 32 ? N - g0 : 32);

#pragma unroll
    for (int k = 0; k < kAccScalars + kShRow; ++k) s_acc[k][tid] = 0.f;
    if (staged) stage_sh_rows(P.sh + g0 * row, nrows, row, lane, s_sh[w]);

    // per-Gaussian forward quantities
    float mx = 0.f, my = 0.f, mz = 0.f, s[3] = {1.f, 1.f, 1.f}, r[9], M[9], Sg6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float qw = 1.f, qx = 0.f, qy = 0.f, qz = 0.f, qi = 1.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) r[i] = M[i] = 0.f;
    if (valid) {
        mx = P.means[3 * g];
        my = P.means[3 * g + 1];
        mz = P.means[3 * g + 2];
        const float *ls = P.log_scales + 3 * g;
        s[0] = expf(ls[0]);
        s[1] = expf(ls[1]);
        s[2] = expf(ls[2]);
        const float *q = P.quats + 4 * g;
        const float qnorm = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        qi = 1.f / qnorm;
        qw = q[0] * qi;
        qx = q[1] * qi;
        qy = q[2] * qi;
        qz = q[3] * qi;
        r[0] = 1.f - 2.f * (qy * qy + qz * qz);
        r[1] = 2.f * (qx * qy - qw * qz);
        r[2] = 2.f * (qx * qz + qw * qy);
        r[3] = 2.f * (qx * qy + qw * qz);
        r[4] = 1.f - 2.f * (qx * qx + qz * qz);
        r[5] = 2.f * (qy * qz - qw * qx);
        r[6] = 2.f * (qx * qz - qw * qy);
        r[7] = 2.f * (qy * qz + qw * qx);
        r[8] = 1.f - 2.f * (qx * qx + qy * qy);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) M[3 * i + j] = r[3 * i + j] * s[j];
        int t = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j)
                Sg6[t++] = M[3 * i] * M[3 * j] + M[3 * i + 1] * M[3 * j + 1] + M[3 * i + 2] * M[3 * j + 2];
    }

    // visible pairs of the warp: one ballot per view, prefix counts
    const int n_views = vsp->n_views;
    for (int v0 = 0; v0 < n_views; v0 += 8) {
        uint32_t t8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) t8[j] = (valid && v0 + j < n_views) ? tiles[(size_t)(v0 + j) * N + g] : 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t m = __ballot_sync(0xffffffffu, t8[j] != 0);
            if (lane == 0 && v0 + j < n_views) s_mask[w][v0 + j] = m;
        }
    }
    __syncwarp();
    if (lane == 0) {
        int acc = 0;
        for (int vi = 0; vi < n_views; ++vi) {
            s_pref[w][vi] = acc;
            acc += __popc(s_mask[w][vi]);
        }
        s_pref[w][n_views] = acc;
    }
    __syncthreads(); // accumulators, staged rows and masks are visible to every lane
    const int total = s_pref[w][n_views];

    for (int base = 0; base < total; base += 32) {
        const int p = base + lane;
        const bool has = p < total;
        int vi = 0, src = lane;
        if (has) {
            while (vi + 1 < n_views && s_pref[w][vi + 1] <= p) ++vi;
            src = (int)__fns(s_mask[w][vi], 0, p - s_pref[w][vi] + 1);
        }
        const float gx = __shfl_sync(0xffffffffu, mx, src);
        const float gy = __shfl_sync(0xffffffffu, my, src);
        const float gz = __shfl_sync(0xffffffffu, mz, src);
        float S6[6];
#pragma unroll
        for (int t = 0; t < 6; ++t) S6[t] = __shfl_sync(0xffffffffu, Sg6[t], src);
        // this pair's terms for its owner's accumulators
        float t_sig[6], dm[3] = {0.f, 0.f, 0.f}, dop = 0.f, Y[16], m3[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t < 6; ++t) t_sig[t] = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) Y[k] = 0.f;
        bool active = false;
        GGrad gg;
        if (has) {
            gg = g2d[(size_t)vi * N + (size_t)(g0 + src)];
            active = !(gg.g0.x == 0.f && gg.g0.y == 0.f && gg.g0.z == 0.f && gg.g0.w == 0.f && gg.g1.x == 0.f &&
                       gg.g1.y == 0.f && gg.g1.z == 0.f && gg.g2.x == 0.f && gg.g2.y == 0.f && gg.g2.z == 0.f);
        }
        if (active) {
            const float mx_ = gg.g0.x, my_ = gg.g0.y, mxx = gg.g0.z, mxy = gg.g0.w;
            const float myy = gg.g1.x, ddepth = gg.g1.z;
            dop = gg.g1.y;
            const float drgb[3] = {gg.g2.x, gg.g2.y, gg.g2.z};
            const float Sg[3][3] = {{S6[0], S6[1], S6[2]}, {S6[1], S6[3], S6[4]}, {S6[2], S6[4], S6[5]}};
            const ViewDesc &V = vsp->v[vi];
            const float px = V.R[0] * gx + V.R[1] * gy + V.R[2] * gz + V.t[0];
            const float py = V.R[3] * gx + V.R[4] * gy + V.R[5] * gz + V.t[1];
            const float pz = V.R[6] * gx + V.R[7] * gy + V.R[8] * gz + V.t[2];
            const float iz = 1.f / pz;
            const float xz = px * iz, yz = py * iz;
            const bool clx = xz < -V.limx || xz > V.limx;
            const bool cly = yz < -V.limy || yz > V.limy;
            const float txc = fminf(V.limx, fmaxf(-V.limx, xz));
            const float tyc = fminf(V.limy, fmaxf(-V.limy, yz));
            const float J00 = V.fx * iz, J02 = -V.fx * txc * iz;
            const float J11 = V.fy * iz, J12 = -V.fy * tyc * iz;
            float T[2][3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T[0][j] = J00 * V.R[j] + J02 * V.R[6 + j];
                T[1][j] = J11 * V.R[3 + j] + J12 * V.R[6 + j];
            }
            float ST[2][3]; // Sigma T_i^T
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int rr = 0; rr < 3; ++rr)
                    ST[i][rr] = Sg[rr][0] * T[i][0] + Sg[rr][1] * T[i][1] + Sg[rr][2] * T[i][2];
            const float a = T[0][0] * ST[0][0] + T[0][1] * ST[0][1] + T[0][2] * ST[0][2] + 0.3f;
            const float b = T[0][0] * ST[1][0] + T[0][1] * ST[1][1] + T[0][2] * ST[1][2];
            const float c = T[1][0] * ST[1][0] + T[1][1] * ST[1][1] + T[1][2] * ST[1][2] + 0.3f;
            const float det = a * c - b * b;
            const float id = 1.f / det, id2 = id * id;
            // screen-space gradients from the compositing moments (power =
            // -(A dx^2 + C dy^2)/2 - B dx dy with the conic (A, B, C) = (c, -b, a) / det)
            const float cA = c * id, cB = -b * id, cC = a * id;
            const float du = -(cA * mx_ + cB * my_), dv = -(cC * my_ + cB * mx_);
            const float dA = -0.5f * mxx, dB = -mxy, dC = -0.5f * myy;
            // conic (A, B, C) = (c, -b, a) / det
            const float da = -c * c * id2 * dA + b * c * id2 * dB + (id - a * c * id2) * dC;
            const float dc = (id - a * c * id2) * dA + a * b * id2 * dB - a * a * id2 * dC;
            const float db = 2.f * b * c * id2 * dA + (-id - 2.f * b * b * id2) * dB + 2.f * a * b * id2 * dC;
            // a = T0 Sigma T0^T, b = T0 Sigma T1^T, c = T1 Sigma T1^T
#pragma unroll
            for (int rr = 0; rr < 3; ++rr)
#pragma unroll
                for (int ss = rr; ss < 3; ++ss) {
                    float v = da * T[0][rr] * T[0][ss] + dc * T[1][rr] * T[1][ss] +
                              0.5f * db * (T[0][rr] * T[1][ss] + T[1][rr] * T[0][ss]);
                    // off-diagonal entries collect both symmetric positions
                    if (ss != rr) v *= 2.f;
                    t_sig[rr == 0 ? ss : (rr == 1 ? 2 + ss : 5)] = v;
                }
            float dT[2][3];
#pragma unroll
            for (int rr = 0; rr < 3; ++rr) {
                dT[0][rr] = 2.f * da * ST[0][rr] + db * ST[1][rr];
                dT[1][rr] = db * ST[0][rr] + 2.f * dc * ST[1][rr];
            }
            float dJ00 = 0.f, dJ02 = 0.f, dJ11 = 0.f, dJ12 = 0.f;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                dJ00 += dT[0][j] * V.R[j];
                dJ02 += dT[0][j] * V.R[6 + j];
                dJ11 += dT[1][j] * V.R[3 + j];
                dJ12 += dT[1][j] * V.R[6 + j];
            }
            const float iz2 = iz * iz;
            float dpx = 0.f, dpy = 0.f, dpz = 0.f;
            dpz -= (dJ00 * V.fx + dJ11 * V.fy) * iz2;
            if (clx) {
                dpz += dJ02 * V.fx * txc * iz2;
            } else {
                dpx -= dJ02 * V.fx * iz2;
                dpz += dJ02 * 2.f * V.fx * px * iz2 * iz;
            }
            if (cly) {
                dpz += dJ12 * V.fy * tyc * iz2;
            } else {
                dpy -= dJ12 * V.fy * iz2;
                dpz += dJ12 * 2.f * V.fy * py * iz2 * iz;
            }
            // screen position and depth
            dpx += du * V.fx * iz;
            dpy += dv * V.fy * iz;
            dpz += -(du * V.fx * px + dv * V.fy * py) * iz2 + ddepth;
#pragma unroll
            for (int k = 0; k < 3; ++k) dm[k] = V.R[k] * dpx + V.R[3 + k] * dpy + V.R[6 + k] * dpz;
            // colour through the SH basis at the view direction
            float ex = gx - V.campos[0], ey = gy - V.campos[1], ez = gz - V.campos[2];
            const float len = sqrtf(ex * ex + ey * ey + ez * ez);
            const float il = 1.f / len;
            ex *= il;
            ey *= il;
            ez *= il;
            sh_values(deg, ex, ey, ez, Y);
            const float *shg = staged ? &s_sh[w][src * kShPitch] : P.sh + (size_t)(g0 + src) * row;
            float w16[16];
            // colour channels clamped at 0 pass no gradient: from the clamp word
            // the forward left in the record, else from the colour re-evaluated
            const uint32_t clamp = __float_as_uint(gg.g2.w);
            if (clamp & kClampKnown) {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) m3[ch] = (clamp >> ch) & 1u ? 0.f : drgb[ch];
            } else {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    float raw = 0.5f;
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        if (k < nk) raw += Y[k] * shg[3 * k + ch];
                    m3[ch] = raw < 0.f ? 0.f : drgb[ch];
                }
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                w16[k] = 0.f;
                if (k < nk) {
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) w16[k] += m3[ch] * shg[3 * k + ch];
                }
            }
            const float3 gd = sh_weighted_grad(deg, ex, ey, ez, w16);
            const float dd = gd.x * ex + gd.y * ey + gd.z * ez;
            dm[0] += (gd.x - ex * dd) * il;
            dm[1] += (gd.y - ey * dd) * il;
            dm[2] += (gd.z - ez * dd) * il;
        }
        // Add the terms to the owner's accumulators with plain read-modify-writes:
        // lanes whose owner also appears at a lower lane of this round wait for
        // their turn, so no two lanes update one column at once.
        const unsigned same = __match_any_sync(0xffffffffu, active ? src : 32 + lane);
        const int turn = __popc(same & ((1u << lane) - 1u));
        const int turns = __reduce_max_sync(0xffffffffu, (unsigned)turn) + 1;
        float *acc_col = &s_acc[0][wbase + src];
        constexpr int ld = kBwdThreads + 1;
        for (int j = 0; j < turns; ++j) {
            if (active && turn == j) {
#pragma unroll
                for (int k = 0; k < 3; ++k) acc_col[ld * k] += dm[k];
#pragma unroll
                for (int t = 0; t < 6; ++t) acc_col[ld * (3 + t)] += t_sig[t];
                acc_col[ld * 9] += dop;
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k < nk) {
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch) acc_col[ld * (kAccScalars + 3 * k + ch)] += Y[k] * m3[ch];
                    }
            }
            __syncwarp();
        }
    }
    __syncwarp();

    if (valid) {
        const float dSig[6] = {s_acc[3][tid], s_acc[4][tid], s_acc[5][tid], s_acc[6][tid], s_acc[7][tid],
                               s_acc[8][tid]};
        const float d_mean[3] = {s_acc[0][tid], s_acc[1][tid], s_acc[2][tid]};
        const float d_op = s_acc[9][tid];
        // dL/dSigma as a symmetric matrix G, seen in the Gaussian's own frame:
        // Gb = R^T G R.  Sigma = R diag(s^2) R^T (Eq. 2), so
        //   dL/d log s_j = 2 s_j^2 Gb_jj,
        // and a rotation dR = [w]x R changes L by -2 c . w, where [c]x is the
        // commutator Sigma G - G Sigma = R [diag(s^2), Gb] R^T, whose entries
        // in the own frame are (s_i^2 - s_j^2) Gb_ij.  The chain rule through
        // R(q) and the normalisation gives the same gradient, but forms it as
        // a large radial part minus its projection; for a nearly isotropic
        // Gaussian that difference cancels most digits of a binary32 result.
        // Here the small factors s_i^2 - s_j^2 are formed directly (exactly
        // for close scales), so each component keeps binary32 accuracy
        // relative to the rotation gradient itself.
        float dS[3][3];
        dS[0][0] = dSig[0];
        dS[1][1] = dSig[3];
        dS[2][2] = dSig[5];
        dS[0][1] = dS[1][0] = 0.5f * dSig[1];
        dS[0][2] = dS[2][0] = 0.5f * dSig[2];
        dS[1][2] = dS[2][1] = 0.5f * dSig[4];
        float GR[3][3]; // G R
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                GR[i][j] = dS[i][0] * r[j] + dS[i][1] * r[3 + j] + dS[i][2] * r[6 + j];
        float Gb[3][3]; // R^T G R
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                Gb[i][j] = r[i] * GR[0][j] + r[3 + i] * GR[1][j] + r[6 + i] * GR[2][j];
        float d_ls[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) d_ls[j] = 2.f * s[j] * s[j] * Gb[j][j];
        // own-frame c, then world frame c = R c_own
        const float c0 = (s[2] - s[1]) * (s[2] + s[1]) * Gb[2][1];
        const float c1 = (s[0] - s[2]) * (s[0] + s[2]) * Gb[0][2];
        const float c2 = (s[1] - s[0]) * (s[1] + s[0]) * Gb[1][0];
        const float cw0 = r[0] * c0 + r[1] * c1 + r[2] * c2;
        const float cw1 = r[3] * c0 + r[4] * c1 + r[5] * c2;
        const float cw2 = r[6] * c0 + r[7] * c1 + r[8] * c2;
        // unit quaternion (w, v): a world rotation w moves it by (0, w) (x) q / 2,
        // so the gradient is -4 [-v . c ; w c - v x c], divided by |q| for the
        // unnormalised parameter
        float dqt[4];
        dqt[0] = -(qx * cw0 + qy * cw1 + qz * cw2);
        dqt[1] = qw * cw0 - (qy * cw2 - qz * cw1);
        dqt[2] = qw * cw1 - (qz * cw0 - qx * cw2);
        dqt[3] = qw * cw2 - (qx * cw1 - qy * cw0);
        const float o = 1.f / (1.f + expf(-P.opacity_logits[g]));
        // the compositing backward accumulates o dL/do (its exponent holds log2 o)
        const float d_logit = d_op * (1.f - o);
        if (!G.accumulate) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                G.d_means[3 * g + k] = d_mean[k];
                G.d_log_scales[3 * g + k] = d_ls[k];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) G.d_quats[4 * g + k] = -4.f * dqt[k] * qi;
            G.d_opacity_logits[g] = d_logit;
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                G.d_means[3 * g + k] += d_mean[k];
                G.d_log_scales[3 * g + k] += d_ls[k];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) G.d_quats[4 * g + k] += -4.f * dqt[k] * qi;
            G.d_opacity_logits[g] += d_logit;
        }
    }
    // SH gradient rows of the warp's Gaussians, contiguous in memory: written
    // with consecutive lanes on consecutive floats
    float *dst = G.d_sh + g0 * row;
    if (row == kShRow) write_sh_grad_rows<kShRow>(dst, nrows, row, 3 * nk, s_acc[kAccScalars], kBwdThreads + 1,
                                                  wbase, lane, G.accumulate);
    else write_sh_grad_rows<0>(dst, nrows, row, 3 * nk, s_acc[kAccScalars], kBwdThreads + 1, wbase, lane,
                               G.accumulate);
}

__global__ void exp_key_kernel(const float *__restrict__ x, float *__restrict__ y, int64_t n, ExpKeyTable t) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = exp_key(x[i], t);
}

// Table and constants of exp_key, from binary64 host arithmetic.
ExpKeyTable make_exp_key_table() {
    ExpKeyTable t;
    for (int j = 0; j < 32; ++j) {
        const double v = std::exp2(j / 32.0);
        t.hi[j] = (float)v;
        t.lo[j] = (float)(v - (double)t.hi[j]);
    }
    const double step = std::log(2.0) / 32.0;
    auto trunc12 = [](double v) {
        int e = 0;
        const double m = std::frexp(v, &e);
        return std::ldexp(std::floor(std::ldexp(m, 12)), e - 12);
    };
    const double c1 = trunc12(step), c2 = trunc12(step - c1);
    t.inv_step = (float)(1.0 / step);
    t.c1 = (float)c1;
    t.c2 = (float)c2;
    t.c3 = (float)(step - c1 - c2);
    return t;
}

const ExpKeyTable &exp_key_table() {
    static const ExpKeyTable t = make_exp_key_table();
    return t;
}

} // namespace

void launch_exp_key(const float *x, float *y, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    int64_t blocks = (n + 255) / 256;
    if (blocks > device_sm_count() * 16) blocks = device_sm_count() * 16;
    exp_key_kernel<<<(unsigned)blocks, 256, 0, s>>>(x, y, n, exp_key_table());
}

void launch_preprocess_fwd(const GaussParams &P, const ViewSet *vs, GRec *recs, uint32_t *tiles,
                           uint32_t *zbits, uint2 *rects, GGrad *g2d_init, cudaStream_t s) {
    if (P.n <= 0) return;
    const int blocks = (P.n + kFwdThreads - 1) / kFwdThreads;
    preprocess_fwd_kernel<<<blocks, kFwdThreads, 0, s>>>(P, vs, recs, tiles, zbits, rects, g2d_init,
                                                         exp_key_table());
}

void launch_preprocess_bwd(const GaussParams &P, const ViewSet *vs, const uint32_t *tiles,
                           const GGrad *g2d, const ParamGrads &G, cudaStream_t s) {
    if (P.n <= 0) return;
    // the dynamic shared-memory limit is raised once per device
    static uint64_t attr_set = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !((attr_set >> dev) & 1u)) {
        cudaFuncSetAttribute(preprocess_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
        attr_set |= (uint64_t)1 << dev;
    }
    const int blocks = (P.n + kBwdThreads - 1) / kBwdThreads;
    preprocess_bwd_kernel<<<blocks, kBwdThreads, kBwdSmem, s>>>(P, vs, tiles, g2d, G);
}

} // namespace lvigs
