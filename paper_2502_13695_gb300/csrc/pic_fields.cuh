// Fused field pass on sm_103a: B half step, E step with the Lorentz
// polarisation current and the Silver-Mueller z faces, B half step, the
// cell-centred |E| window and the Keldysh cache check, in one kernel.
//
// Each CTA owns an (x, y) tile of FTX x FTY points and a chunk of FZ z planes
// and marches up the chunk.  Shared memory holds three planes of E^n, two of
// B^{n+1/2} and two of E^{n+1}, each with the halo the next stage needs:
//   B^{n+1} on the tile     needs E^{n+1} on tile + (1, 1)
//   E^{n+1} on tile + (1,1) needs B^{n+1/2} on tile + (-1..1, -1..1)
//   B^{n+1/2} there         needs E^n on tile + (-1..2, -1..2)
// and along z B^{n+1/2}(k) needs E^n(k+1), E^{n+1}(k) needs B^{n+1/2}(k-1),
// B^{n+1}(k) and the window of cell k need E^{n+1}(k+1).  Halo points are
// recomputed redundantly, so the pass reads E, B, J, P, Q from the current
// buffers and writes the owned points of the other buffers (double
// buffering); J of the other buffer is cleared for the next deposit.
// Global inputs move to shared memory with cp.async one plane iteration
// ahead (E^n(q+3), B^n(q+2), J, P, Q(q+2) while plane q is computed), into
// double-buffered staging, so DRAM latency overlaps a whole plane of work.
#pragma once
#include "pic_kernels.cuh"

namespace pg {

constexpr int FTX = 32, FTY = 16, FZ = 32, FTHREADS = 256;
constexpr int FEX = FTX + 3, FEY = FTY + 3;  // E^n region, origin (x0-1, y0-1)
constexpr int FBX = FTX + 2, FBY = FTY + 2;  // B^{n+1/2} region, same origin
constexpr int FFX = FTX + 1, FFY = FTY + 1;  // E^{n+1} region, origin (x0, y0)
constexpr int FEP = FEX * FEY, FBP = FBX * FBY, FFP = FFX * FFY;
// shared memory, in reals: E^n ring (3 planes x 3), B^n staging (2 x 3),
// J staging (2 x 4 interleaved), P, Q staging (2 x 6), B^{n+1/2} (2 x 3),
// E^{n+1} (2 x 3)
// (every region starts on a multiple of 4 reals: 16-byte cp.async needs
// 16-byte aligned shared addresses)
constexpr int fsm_al(int x) { return (x + 3) & ~3; }
constexpr int FSM_EN = 0;
constexpr int FSM_BN = fsm_al(FSM_EN + 9 * FEP);
constexpr int FSM_J = fsm_al(FSM_BN + 6 * FBP);
constexpr int FSM_PQ = fsm_al(FSM_J + 8 * FFP);
constexpr int FSM_BH = fsm_al(FSM_PQ + 12 * FFP);
constexpr int FSM_E1 = fsm_al(FSM_BH + 6 * FBP);
constexpr int FSMEM_ELEMS = fsm_al(FSM_E1 + 6 * FFP);
static_assert(FSM_J % 4 == 0 && (4 * FFP) % 4 == 0, "J staging must be 16-byte aligned");

// Where the field pass writes (the non-current halves of the double buffers).
template <class R>
struct FieldOut {
  R *E[3], *B[3], *P[3], *Q[3];
  R *Jclear;
};

template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(gmem), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <class R>
__device__ __forceinline__ void window_update(const Ctx<R> &X, long long m, int k, R a) {
  const Dev<R> &D = X.d;
  const int NW = D.NW;
  const int s = (int)(*D.step % NW);
  R *__restrict__ W = D.win + m;
  const long long st = D.nmat;
  W[s * st] = a;
  const R pm = s == 0 ? a : fmax(D.pm[m], a);
  D.pm[m] = pm;
  const R amp = s + 1 < NW ? fmax(pm, W[(s + 1) * st]) : pm;
  if (s == NW - 1) {
    R run = W[(NW - 1) * st];
    for (int q = NW - 2; q >= 0; --q) {
      run = fmax(run, W[q * st]);
      W[q * st] = run;
    }
  }
  D.eamp[m] = amp;
  bool need = false;
  if (D.ckey[m] != amp) {
    const LayerR<R> &L = X.lr[D.layer_of_plane[k]];
    if (!(amp >= L.e_skip)) {
      D.T[m] = 0ull;
      D.ckey[m] = amp;
    } else {
      need = true;
    }
  }
  const unsigned act = __activemask();
  const unsigned want = __ballot_sync(act, need);
  if (need) {
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(want) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(X.work_n, __popc(want));
    base = __shfl_sync(want, base, leader);
    X.work[base + __popc(want & ((1u << lane) - 1u))] = (int)m;
  }
}

template <class R>
__global__ void __launch_bounds__(FTHREADS) k_fields(Ctx<R> X, FieldOut<R> W, int do_window) {
  const Dev<R> &D = X.d;
  extern __shared__ __align__(16) unsigned char fsm_raw[];
  R *const sm = reinterpret_cast<R *>(fsm_raw);
  R *const En = sm + FSM_EN;  // [3 slots][3][FEP]
  R *const Bn = sm + FSM_BN;  // [2 slots][3][FBP]
  R *const Js = sm + FSM_J;   // [2 slots][FFP][4]
  R *const PQ = sm + FSM_PQ;  // [2 slots][6][FFP]
  R *const Bh = sm + FSM_BH;  // [2 slots][3][FBP]
  R *const E1 = sm + FSM_E1;  // [2 slots][3][FFP]
  const int nx = D.nx, ny = D.ny, nz = D.nz, nxy = D.nxy;
  const int ntx = (nx + FTX - 1) / FTX, nty = (ny + FTY - 1) / FTY;
  int bid = blockIdx.x;
  const int tix = bid % ntx;
  bid /= ntx;
  const int tiy = bid % nty;
  const int kc = bid / nty;
  const int x0 = tix * FTX, y0 = tiy * FTY;
  const int txe = min(FTX, nx - x0), tye = min(FTY, ny - y0);
  const int k0 = kc * FZ, k1 = min(k0 + FZ, nz + 1);
  const R h = R(0.5) * D.dt;
  const R idx = D.idx, idy = D.idy, idz = D.idz;
  const R c2dt = D.c2dt, dtie = R(D.dt_d / kEps0);
  const int tid = threadIdx.x;
  R joule = R(0);

  auto wx = [&](int x) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); };
  auto wy = [&](int y) { return y < 0 ? y + ny : (y >= ny ? y - ny : y); };
  auto slotE = [](int k) { return ((k % 3) + 3) % 3; };

  // asynchronous staging of plane k's inputs (nothing for planes outside 0..nz)
  auto stage_En = [&](int k) {
    if (k < 0 || k > nz) return;
    R *dst = En + slotE(k) * 3 * FEP;
    const int w = txe + 3, n = w * (tye + 3);
    for (int q = tid; q < n; q += FTHREADS) {
      const int ly = q / w, lx = q - ly * w;
      const long long o = (long long)k * nxy + wy(y0 - 1 + ly) * nx + wx(x0 - 1 + lx);
      const int l = ly * FEX + lx;
      cp_async<sizeof(R)>(dst + l, D.E[0] + o);
      cp_async<sizeof(R)>(dst + FEP + l, D.E[1] + o);
      cp_async<sizeof(R)>(dst + 2 * FEP + l, D.E[2] + o);
    }
  };
  auto stage_Bn = [&](int k) {
    if (k < 0 || k > nz) return;
    R *dst = Bn + (k & 1) * 3 * FBP;
    const int w = txe + 2, n = w * (tye + 2);
    for (int q = tid; q < n; q += FTHREADS) {
      const int ly = q / w, lx = q - ly * w;
      const long long o = (long long)k * nxy + wy(y0 - 1 + ly) * nx + wx(x0 - 1 + lx);
      const int l = ly * FBX + lx;
      if (k < nz) {
        cp_async<sizeof(R)>(dst + l, D.B[0] + o);
        cp_async<sizeof(R)>(dst + FBP + l, D.B[1] + o);
      }
      cp_async<sizeof(R)>(dst + 2 * FBP + l, D.B[2] + o);
    }
  };
  auto stage_JPQ = [&](int k) {
    if (k < 0 || k > nz) return;
    R *js = Js + (k & 1) * 4 * FFP;
    R *pq = PQ + (k & 1) * 6 * FFP;
    const int L = k < nz ? D.layer_of_plane[k] : -1;
    const int w = txe + 1, n = w * (tye + 1);
    for (int q = tid; q < n; q += FTHREADS) {
      const int ly = q / w, lx = q - ly * w;
      const int r = wy(y0 + ly) * nx + wx(x0 + lx);
      const long long o = (long long)k * nxy + r;
      const int l = ly * FFX + lx;
      if (sizeof(R) == 4) {
        cp_async<16>(js + 4 * l, D.J4 + 4 * o);
      } else {
        cp_async<16>(js + 4 * l, D.J4 + 4 * o);
        cp_async<16>(js + 4 * l + 2, D.J4 + 4 * o + 2);
      }
      if (L >= 0) {
        const long long m = (long long)D.mplane[k] * nxy + r;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          cp_async<sizeof(R)>(pq + d * FFP + l, D.P[d] + m);
          cp_async<sizeof(R)>(pq + (3 + d) * FFP + l, D.Q[d] + m);
        }
      }
    }
  };

  // B^{n+1/2}(k) on the region (txe+2) x (tye+2), same origin as E^n
  auto half_B = [&](int k) {
    const R *e0 = En + slotE(k) * 3 * FEP;
    const R *e1 = (k < nz) ? En + slotE(k + 1) * 3 * FEP : nullptr;
    const R *bn = Bn + (k & 1) * 3 * FBP;
    R *dst = Bh + (k & 1) * 3 * FBP;
    const int w = txe + 2, n = w * (tye + 2);
    for (int q = tid; q < n; q += FTHREADS) {
      const int ly = q / w, lx = q - ly * w;
      const int l = ly * FEX + lx;
      const int lb = ly * FBX + lx;
      const R ex = e0[l], ey = e0[FEP + l], ez = e0[2 * FEP + l];
      R bx = R(0), by = R(0);
      if (k < nz) {
        bx = bn[lb] - h * ((e0[2 * FEP + l + FEX] - ez) * idy - (e1[FEP + l] - ey) * idz);
        by = bn[FBP + lb] - h * ((e1[l] - ex) * idz - (e0[2 * FEP + l + 1] - ez) * idx);
      }
      const R bz = bn[2 * FBP + lb] - h * ((e0[FEP + l + 1] - ey) * idx - (e0[l + FEX] - ex) * idy);
      dst[lb] = bx;
      dst[FBP + lb] = by;
      dst[2 * FBP + lb] = bz;
    }
  };

  // E^{n+1}(k) on the region (txe+1) x (tye+1), origin (x0, y0); owned points
  // (inside the tile and the chunk) are written to the output buffers
  auto full_E = [&](int k) {
    const R *e0 = En + slotE(k) * 3 * FEP;
    const R *b0 = Bh + (k & 1) * 3 * FBP;
    const R *bm = (k > 0) ? Bh + ((k - 1) & 1) * 3 * FBP : nullptr;
    const R *js = Js + (k & 1) * 4 * FFP;
    const R *pq = PQ + (k & 1) * 6 * FFP;
    R *dst = E1 + (k & 1) * 3 * FFP;
    const int L = k < nz ? D.layer_of_plane[k] : -1;
    const bool own_plane = k >= k0 && k < k1;
    R exi = R(0), eyi = R(0);
    if (k == 0) {
      const double t = ((double)(*D.step) + 0.5) * D.dt_d - D.t_peak;
      const double env = exp(-2.0 * 0.69314718055994531 * t * t / (D.fwhm * D.fwhm));
      const double einc = D.E0 * env * cos(D.omega * t + D.cep);
      exi = D.pol == 0 ? R(einc) : R(0);
      eyi = D.pol == 0 ? R(0) : R(einc);
    }
    const int w = txe + 1, n = w * (tye + 1);
    for (int q = tid; q < n; q += FTHREADS) {
      const int ly = q / w, lx = q - ly * w;
      const int le = (ly + 1) * FEX + (lx + 1);  // in the E^n frame
      const int lb = (ly + 1) * FBX + (lx + 1);  // in the B^{n+1/2} frame
      const int lf = ly * FFX + lx;
      const bool own = own_plane && lx < txe && ly < tye;
      const R jx = js[4 * lf], jy = js[4 * lf + 1], jz = js[4 * lf + 2];
      const R bz = b0[2 * FBP + lb];
      const R dBz_dy = (bz - b0[2 * FBP + lb - FBX]) * idy;
      const R dBz_dx = (bz - b0[2 * FBP + lb - 1]) * idx;
      const R ex0 = e0[le], ey0 = e0[FEP + le], ez0 = e0[2 * FEP + le];
      R ex1, ey1, ez1 = R(0);
      R px = R(0), py = R(0), pz = R(0), qx = R(0), qy = R(0), qz = R(0);
      if (L >= 0) {
        px = pq[lf];
        py = pq[FFP + lf];
        pz = pq[2 * FFP + lf];
        qx = pq[3 * FFP + lf];
        qy = pq[4 * FFP + lf];
        qz = pq[5 * FFP + lf];
      }
      if (k == 0 || k == nz) {
        const R al = D.alpha, cc = R(kC);
        const R inv = R(1) / (R(1) + al);
        if (k == 0) {
          ex1 = ((R(1) - al) * ex0 - R(2) * al * cc * b0[FBP + lb] + R(4) * al * exi +
                 (c2dt * dBz_dy - dtie * jx)) * inv;
          ey1 = ((R(1) - al) * ey0 + R(2) * al * cc * b0[lb] + R(4) * al * eyi -
                 (c2dt * dBz_dx + dtie * jy)) * inv;
        } else {
          ex1 = ((R(1) - al) * ex0 + R(2) * al * cc * bm[FBP + lb] + (c2dt * dBz_dy - dtie * jx)) * inv;
          ey1 = ((R(1) - al) * ey0 - R(2) * al * cc * bm[lb] - (c2dt * dBz_dx + dtie * jy)) * inv;
        }
      } else {
        const R ax = c2dt * (dBz_dy - (b0[FBP + lb] - bm[FBP + lb]) * idz) - dtie * jx;
        const R ay = c2dt * ((b0[lb] - bm[lb]) * idz - dBz_dx) - dtie * jy;
        if (L >= 0) {
          const LayerR<R> &Ly = X.lr[L];
          ex1 = e_point(Ly, ex0, ax, px, qx);
          ey1 = e_point(Ly, ey0, ay, py, qy);
        } else {
          ex1 = ex0 + ax;
          ey1 = ey0 + ay;
        }
      }
      if (k < nz) {
        const R az = c2dt * ((b0[FBP + lb] - b0[FBP + lb - 1]) * idx - (b0[lb] - b0[lb - FBX]) * idy) -
                     dtie * jz;
        if (L >= 0)
          ez1 = e_point(X.lr[L], ez0, az, pz, qz);
        else
          ez1 = ez0 + az;
      }
      dst[lf] = ex1;
      dst[FFP + lf] = ey1;
      dst[2 * FFP + lf] = ez1;
      if (own) {
        const int r = (y0 + ly) * nx + (x0 + lx);
        const long long o = (long long)k * nxy + r;
        W.E[0][o] = ex1;
        W.E[1][o] = ey1;
        W.E[2][o] = ez1;
        if (L >= 0) {
          const long long m = (long long)D.mplane[k] * nxy + r;
          W.P[0][m] = px;
          W.P[1][m] = py;
          W.P[2][m] = pz;
          W.Q[0][m] = qx;
          W.Q[1][m] = qy;
          W.Q[2][m] = qz;
        }
        clear_j3(W.Jclear + 4 * o);
        joule += jx * R(0.5) * (ex0 + ex1) + jy * R(0.5) * (ey0 + ey1) + jz * R(0.5) * (ez0 + ez1);
      }
    }
  };

  // B^{n+1}(k) and the window of cell k on the owned tile
  auto finish = [&](int k) {
    const R *f0 = E1 + (k & 1) * 3 * FFP;
    const R *f1 = (k < nz) ? E1 + ((k + 1) & 1) * 3 * FFP : nullptr;
    const R *b0 = Bh + (k & 1) * 3 * FBP;
    const bool mat = do_window && k < nz && D.layer_of_plane[k] >= 0;
    const int n = txe * tye;
    for (int q = tid; q < n; q += FTHREADS) {
      const int ly = q / txe, lx = q - ly * txe;
      const int lf = ly * FFX + lx;
      const int lb = (ly + 1) * FBX + (lx + 1);
      const int r = (y0 + ly) * nx + (x0 + lx);
      const long long o = (long long)k * nxy + r;
      const R ex = f0[lf], ey = f0[FFP + lf], ez = f0[2 * FFP + lf];
      R bx = R(0), by = R(0);
      if (k < nz) {
        bx = b0[lb] - h * ((f0[2 * FFP + lf + FFX] - ez) * idy - (f1[FFP + lf] - ey) * idz);
        by = b0[FBP + lb] - h * ((f1[lf] - ex) * idz - (f0[2 * FFP + lf + 1] - ez) * idx);
      }
      const R bz = b0[2 * FBP + lb] - h * ((f0[FFP + lf + 1] - ey) * idx - (f0[lf + FFX] - ex) * idy);
      W.B[0][o] = bx;
      W.B[1][o] = by;
      W.B[2][o] = bz;
      if (mat) {
        // |E| at the cell centre from the mean of the 4 edges of each component
        const R ax = R(0.25) * (((f0[lf] + f0[lf + FFX]) + f1[lf]) + f1[lf + FFX]);
        const R ay = R(0.25) * (((f0[FFP + lf] + f0[FFP + lf + 1]) + f1[FFP + lf]) + f1[FFP + lf + 1]);
        const R az = R(0.25) * (((f0[2 * FFP + lf] + f0[2 * FFP + lf + 1]) + f0[2 * FFP + lf + FFX]) +
                                f0[2 * FFP + lf + FFX + 1]);
        const R a = sqrt(ax * ax + ay * ay + az * az);
        window_update(X, (long long)D.mplane[k] * nxy + r, k, a);
      }
    }
  };

  // prologue: E^n(k0-1 .. k0+1), B^{n+1/2}(k0-1, k0), E^{n+1}(k0)
  stage_En(k0 - 1);
  stage_En(k0);
  stage_En(k0 + 1);
  stage_Bn(k0 - 1);
  stage_Bn(k0);
  stage_JPQ(k0);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  if (k0 >= 1) half_B(k0 - 1);
  half_B(k0);
  __syncthreads();
  full_E(k0);
  __syncthreads();
  // inputs of the first loop iteration
  stage_En(k0 + 2);
  stage_Bn(k0 + 1);
  stage_JPQ(k0 + 1);
  cp_async_commit();
  for (int q = k0; q < k1; ++q) {
    cp_async_wait_all();  // E^n(q+2), B^n(q+1), J/P/Q(q+1) have landed
    __syncthreads();
    if (q + 1 < k1) {      // next plane's inputs, in flight during this one
      stage_En(q + 3);
      stage_Bn(q + 2);
      stage_JPQ(q + 2);
    }
    cp_async_commit();
    if (q + 1 <= nz) half_B(q + 1);
    __syncthreads();
    if (q + 1 <= nz) full_E(q + 1);
    __syncthreads();
    finish(q);
  }
  cp_async_wait_all();
  const R tot = block_sum_r(joule);
  if (threadIdx.x == 0 && tot != R(0)) atomicAdd(D.acc + 0, (double)tot * D.dt_d * D.V_d);
}

}  // namespace pg
