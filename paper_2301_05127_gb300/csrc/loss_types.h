// Launch descriptors shared by the host runtime (loss_api.cu) and the kernels (loss_kernels*.cu).
// Plain structs passed by value as kernel parameters.
#pragma once

#include <cstdint>

namespace lossk {

// How one thread block's bundle of whole lines along one axis maps to a field array.
//   X flavour: lines along the contiguous axis; bundle b holds rows r = b*L .. b*L + L - 1 of the flattened
//              (z, y) row index; row r starts at (r / ny1) * sz + (r % ny1) * sy.
//   S flavour: lines along a strided axis; bundle b = outer * nxb + xb holds the L neighbouring x positions
//              x0 = xb * L ..; line l starts at outer * so + x0 + l and steps by pstride.
struct LineGeom {
  int n;       // intervals along the axis (n + 1 points per line)
  int p, M;    // patches and patch length
  int NC;      // chunks per patch
  int n_nb;    // PMBC halo width
  int L;       // lines per bundle
  int pitch;   // shared-memory pitch (X: per line, S: per position)
  int buf;     // elements per shared-memory line buffer (padded layout used by the solve)
  int stage;   // elements per shared-memory staging buffer (dense rows of `spitch`, X flavour only)
  int spitch;  // staging row pitch (n + 1 rounded up to 16 bytes)
  unsigned mmagic;  // ceil(2^32 / M)
  int nbundles;
  // X flavour
  int ny1;
  int64_t sz, sy;
  int64_t nrows;
  // S flavour
  int nx1, nxb;
  int64_t so, pstride;
};

struct Tables {
  const double* W;    // PMBC weights [(p+1)][2 n_nb + 1], scaled by h/3
  const float* t32;   // Thomas factors m_j, j < 64
  const double* t64;
};

template <typename T>
struct DerivArgs {
  LineGeom g;
  Tables tb;
  const T* f;
  T* d1;
  T* d2;
  double* phi_out;
  T s1;     // 3 / h
  double s1d;  // 3 / h in double (phi output)
  T s2;     // 6 / h^2
  T minf;   // 2 - sqrt(3)
  int lines_per_outer;  // S flavour: lines per outer index in the phi_out ordering (= nx1)
};

// Largest block of the persistent batched kernels.
constexpr int kBatchThreads = 512;

// Tile geometry of the FP32 truncated-convolution kernels (loss_kernels_tiled.cu): derivative axis of n intervals
// in p patches of M, halo H positions per side, ntl tiles across the other axis (z tiles: groups of 32 columns,
// x tiles: groups of R rows), ncross points along the other axis, row pitch px; W = PMBC weights of the axis
// (scaled by h/3); r, a, rho = r^M and inv = 1 / (1 - rho^2) of loss_fir.cuh.
struct TileGeom {
  int n, p, M, n_nb, H, ntl, R, ncross;
  int64_t px;
  const double* W;
  const double* Wd;  // junction-correction weights [(p + 1)][2 Rd + 1] (PMBC weights minus convolution weights)
  int Rd;            // their half width, max(n_nb, K)
  int pw;            // absorbing-layer width along the axis (0 = no layer)
  float s3h, r, a, rho, inv;
  float s3h_lo;      // rounding error of s3h (mulc)
};

// Device-side step counters of one shot, used by launches whose arguments do not change from step to step
// (persistent batched launches and captured CUDA graphs): step = index n of the step being taken, row = trace row
// the step's receiver values go to; both advance once per step (row by row_inc, 1 when the shot records).
struct StepClock {
  int64_t step;
  int64_t row;
  int64_t row_inc;
  int64_t pad;
};

struct SourceArgs {
  int on;
  int zs, ys, xs;    // centre
  double amp;        // dt * amp * f_r(t) / (sum of profile * cell volume), or 0
  double g[25];      // exp(-o^2 / 8), o = -12..12
  // When amp_tab is set, the amplitude of step n is amp_tab[clk->step] (same host-computed values as amp).
  const double* amp_tab;
  const StepClock* clk;
};

// One receiver gather of a batched launch: out row = trace + clk->row * n_rcv + off (see k_gather for modes).
template <typename T>
struct GatherJob {
  const T* f;
  const int64_t* idx;
  int64_t cnt;
  T* trace;
  int64_t n_rcv;
  int64_t off;
  const T* d[3];
  const StepClock* clk;
  int mode;
  int pad;
};

// Exponential-flow coefficients of the ADE-PML along one axis for one step length tau (paper Sec. 3.3):
// tab[0][i] = E = exp(-beta tau), tab[1][i] = (d/k^2)(1 - E)/beta, tab[2][i] = 1/beta,
// tab[3][i] = tau alpha / (d + alpha k), for i = 0..n; points with i < width or i > n - width are in the layer.
template <typename T>
struct PmlAxis {
  const T* tab;
  int width;
  int n;
  const T* tabh;  // the same coefficients for tau / 2 (exact integer-time receiver values), or null
  __device__ __forceinline__ bool in(int i) const { return i < width || i > n - width; }
  // Increment factor of the first half (tau / 2) of the sub-step, from the memory value before the step; the
  // memory variable is not changed.  Requires tabh.
  __device__ __forceinline__ T half(const T* mem, int64_t gi, int i, T g) const {
    const int n1 = n + 1;
    const T m0 = mem[gi];
    const T m1 = tabh[i] * m0 - tabh[n1 + i] * g;
    return tabh[2 * n1 + i] * (m1 - m0) - tabh[3 * n1 + i] * g;
  }
  // Advance the memory variable over tau with frozen derivative g; return the field increment factor.
  __device__ __forceinline__ T step(T* mem, int64_t gi, int i, T g) const {
    const int n1 = n + 1;
    const T m0 = mem[gi];
    const T m1 = tab[i] * m0 - tab[n1 + i] * g;
    mem[gi] = m1;
    return tab[2 * n1 + i] * (m1 - m0) - tab[3 * n1 + i] * g;
  }
};

template <typename T>
struct AcXArgs {
  LineGeom g;
  Tables tb;
  T* sigma;
  T* v1;
  const T* kappa;
  const T* b;        // buoyancy 1/rho, or null when constant (then b0)
  T b0;
  const T* tmp;      // d_z v3 at the current half step (read when do_B)
  T* csig;           // Kahan compensation (KAHAN only)
  T* cv1;
  T dt;              // B step length
  T acoef;           // A step length (dt, dt/2 or -dt/2)
  T s3h;             // 3 / h_x
  T dt_lo, acoef_lo, s3h_lo, b0_lo;  // rounding errors of dt, acoef, s3h, b0 (mulc; 0 in FP64)
  T sc, sc_lo;       // -acoef * b0 * s3h and its rounding error (the velocity update with constant density)
  T minf;
  int do_B;
  SourceArgs src;
  int pml;
  PmlAxis<T> xA, xB, zB;  // x layer for the A step length, x and z layers for tau = dt (B)
  T* psix;
  T* phix;
  T* phiz;
  T* dlt;  // v1 receiver correction b (X(dt/2) - X(dt)/2) in the x layers, or null
};

template <typename T>
struct AcZArgs {
  LineGeom g;
  Tables tb;
  const T* sigma;
  T* v3;
  const T* b;        // or null (then b0)
  T b0;
  T* tmp;            // out: d_z v3 after the update (when do_tmp)
  T* cv3;
  T acoef;
  T s3h;             // 3 / h_z
  T acoef_lo, s3h_lo, b0_lo;  // rounding errors (mulc; 0 in FP64)
  T sc, sc_lo;       // -acoef * b0 * s3h and its rounding error
  T minf;
  int do_tmp;
  int pml;
  PmlAxis<T> zA;
  T* psiz;
  T* dlt;  // v3 receiver correction in the z layers, or null
};

// One line pass of the 3-D elastic step (see loss_kernels_elastic.cu).  src: the three fields differentiated
// along the pass axis; fld/cmp: the nine fields and their compensation terms (LOSS_FIELD_* order); tmp: TA..TE
// (stress sub-step, 0..4) and UA..UC (velocity sub-step, 5..7); memB/memA: PML memory variables of the three
// derivative terms of this pass in the stress and velocity sub-steps.
template <typename T>
struct ElArgs {
  LineGeom g;
  Tables tb;
  const T* src[3];
  T* fld[9];
  T* cmp[9];
  T* tmp[8];
  const T* lam;  // or null (then lam0)
  const T* mu;
  const T* b;
  T lam0, mu0, b0;
  T dt, acoef, s3h, minf;
  T dt_lo, acoef_lo, s3h_lo, lam0_lo, mu0_lo, b0_lo;  // rounding errors (mulc; 0 in FP64)
  int do_B, do_A;
  int pml;
  PmlAxis<T> pB, pA;
  T* memB[3];
  T* memA[3];
  T* dlt[3];  // receiver corrections of the three velocity terms of this pass (in its layers), or null
  SourceArgs srcp;
  int src_explosive, src_shear;
  int force_mask;  // body-force components of the source in the A passes: bit i = f_{i+1} (on v_{i+1})
};

// One term of the adjoint of the time step (see loss_kernels_adjoint.cu).  A term is a forward update
// "field += c * Z" with Z = sgn * X and X the (PML) integral over tau of minus the derivative along the line axis
// of the forward field ffwd; the kernel adds D^T gbar to `out`, where gbar is the adjoint of that derivative,
// updates the adjoint memory variable and accumulates the model gradients.
template <typename T>
struct AdjArgs {
  LineGeom g;
  Tables tb;
  T s3h, minf;
  double s3hd;       // 3 / h in double
  int mode;          // 0: out += D^T in3 only; 1: velocity-sub-step term; 2: stress-sub-step term
  T sgn;             // +1 (acoustic: field += c X) or -1 (elastic: field += c (-X))
  T tau;             // sub-step length
  const T* ffwd;     // forward field differentiated along the line axis (modes 1, 2)
  const T* memf;     // forward memory variable of the term before the sub-step (in layers), or null
  T* memb;           // adjoint memory variable of the term (in / out), or null
  int pml;
  PmlAxis<T> pa;     // tables for tau and, for the receiver terms of mode 1, tau / 2 (tabh)
  const T* in[3];    // adjoint inputs weighted by c1 (summed), or null
  const T* in3;      // adjoint input weighted by c2
  const T* rv;       // mode 1: trace residual at velocity receivers (zero elsewhere), or null
  const T* c1;       // coefficient arrays, or null for the scalars c1s / c2s
  const T* c2;
  T c1s, c2s, cw2;   // c2 = cw2 * (c2 array or c2s)
  double* g1;        // gradient of the c1 parameter: += Z * sum(in), or null
  double* g2;        // gradient of the c2 parameter: += Z * gw2 * in3 + Zh * rv, or null
  T gw2;
  T* out;
};

// Receiver residual injection of one adjoint step.  phase 0: stress fields lam[idx] += r, velocity residual
// arrays rv[idx] += r; phase 1: velocity fields lam[idx] += r and rv[idx] = 0.
template <typename T>
struct InjectJob {
  T* lam;
  T* rv;             // velocity receivers only, else null
  const int64_t* idx;
  const double* r;   // residual of this field's receivers for the step
  int64_t cnt;
};

// Dynamic shared memory of k_xp, in floats: 2 stages x NA staged rows of RW floats, the slow chunks' derivative
// values O, the junction-correction weights (FP64), 2 stages x 2 layer segments (F floats each) of the x memory
// variables, the warm-up partial sums PA / PB, and the x layer's coefficient tables (B step, A step, A half step;
// 4 rows of F each).
struct XpSmem {
  int NA, RW, O, WS, SEG, F, PA, PB, TAB, DL, total;
};
// Descriptor of one shot in a batched z launch.
struct TzShot {
  AcZArgs<float> a;
  TileGeom t;
  int nwj;  // warps of the shot's single-shot launch
  int pad;
};

// Descriptor of one shot in a batched x launch: its rows come in units of R consecutive rows, the global units
// unit0 .. unit0 + ceil(t.ncross / R) - 1.
constexpr int kXpMaxGroups = 8;

// Elastic y / z tile passes (FP32 truncated-convolution form).
enum { ET_BY = 0, ET_BZ = 1, ET_AZ = 2, ET_AY = 3 };
struct ElTile {
  TileGeom t;       // the pass axis: n, p, M, H, Rd, Wd, s3h, r, a, rho, inv; t.px = stride along the axis
  int64_t ostride;  // stride of the remaining axis (z for y tiles, y for z tiles)
  int nouter;       // its extent
  int ncg;          // groups of 32 x columns
  int nx;           // x columns
};
struct XpShot {
  AcXArgs<float> a;
  TileGeom t;
  unsigned mmagic;
  int unit0;
  int R;
  int pad;
};

}  // namespace lossk
