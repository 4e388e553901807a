// Launchers of the 3D FFT passes and of the fused spectral operators.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "adjoint.h"
#include "fft_impl.cuh"
#include "fft_tma.cuh"

namespace pmlens {

namespace {

// Kernel attributes and occupancy belong to one device: they are set or
// measured once per device (with that device current), thread-safely.
constexpr int kMaxDevices = 64;

int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) d = 0;
  return d;
}

// resident block slots of a kernel on the current device (blocks per SM x SMs)
template <typename K>
int device_slots(std::once_flag* once, int* vals, K kernel, int threads, size_t smem) {
  const int d = current_device();
  std::call_once(once[d], [&] {
    int per_sm = 0, nsm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, d);
    vals[d] = std::max(per_sm, 1) * std::max(nsm, 1);
  });
  return vals[d];
}

template <typename R, int N>
struct Launch {
  using C = typename CT<R>::T;
  // algorithmic bytes of one pass: real mesh R, unpadded half-spectrum C
  static constexpr double RB = (double)N * N * N * sizeof(R);
  static constexpr double CB = (double)N * N * (N / 2 + 1) * sizeof(C);
  static size_t smem_x() {
    return (size_t)RowTile<R, N>::SMEM;
  }
  static size_t smem_cols() { return (size_t)(N + N * ColTile<R, N>::W) * sizeof(C); }
  static size_t smem_z() { return (size_t)(N + 2 * N * ZTile<R, N>::W) * sizeof(C); }
  static int ntiles() { return (N / 2 + 1 + ColTile<R, N>::W - 1) / ColTile<R, N>::W; }
  using TT = TmaTile<R, N>;
  // persistent TMA column passes: one block per SM slot the occupancy allows
  static int tma_grid(int tiles) {
    static std::once_flag once[kMaxDevices];
    static int slots[kMaxDevices];
    return std::min(tiles, device_slots(once, slots, k_fft_cols_tma<R, N, false, false>, TT::THREADS, TT::SMEM));
  }

  // persistent x c2r: every block slot the occupancy allows
  static int x_grid(int nblk) {
    attrs();
    static std::once_flag once[kMaxDevices];
    static int slots[kMaxDevices];
    return std::min(nblk, device_slots(once, slots, k_fft_x_c2r<R, N>, RowTile<R, N>::THREADS, smem_x()));
  }

  static void attrs() {
    static std::once_flag once[kMaxDevices];
    std::call_once(once[current_device()], set_attrs);
  }
  static void set_attrs() {
    cudaFuncSetAttribute(k_fft_x_r2c<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_x());
    cudaFuncSetAttribute(k_fft_x_c2r<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_x());
    cudaFuncSetAttribute(k_fft_cols<R, N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols());
    cudaFuncSetAttribute(k_fft_cols<R, N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols());
    cudaFuncSetAttribute(k_zpass_op<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_z());
    cudaFuncSetAttribute(k_zpass_op_tma<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, ZTma<R, N>::SMEM);
    cudaFuncSetAttribute(k_zpass_combine<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_z());
    cudaFuncSetAttribute(k_fft_cols_tma<R, N, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TT::SMEM);
    cudaFuncSetAttribute(k_fft_cols_tma<R, N, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, TT::SMEM);
    cudaFuncSetAttribute(k_fft_cols_tma<R, N, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TT::SMEM);
    cudaFuncSetAttribute(k_fft_cols_tma<R, N, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TT::SMEM);
    cudaFuncSetAttribute(k_fft_cols_tma<R, N, true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         TT::SMEM_DUAL);
    if constexpr (std::is_same<R, float>::value) {
      cudaFuncSetAttribute(k_fft_x_r2c_il<N, 4, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           RowTileIL<N, 3>::SMEM);
      cudaFuncSetAttribute(k_fft_x_r2c_il<N, 4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           RowTileIL<N, 4>::SMEM);
      cudaFuncSetAttribute(k_fft_x_r2c_il<N, 2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           RowTileIL<N, 2>::SMEM);
    }
    // an attribute this device refuses would otherwise surface as the error of an unrelated
    // later launch check; a kernel that really needs it fails at its own launch
    cudaGetLastError();
  }

  static void x_fwd(const R* in, C* out, int P, cudaStream_t s, Prof* pf, int kind) {
    ProfScope ps(pf, kind >= 0 ? kind : KK_FFT_X_FWD, s, RB + CB);
    k_fft_x_r2c<R, N><<<(long long)N * N / RowTile<R, N>::ROWS, RowTile<R, N>::THREADS, smem_x(), s>>>(in, out, P);
  }
  static void x_inv(const C* in, R* out, int P, cudaStream_t s, Prof* pf, int kind) {
    ProfScope ps(pf, kind >= 0 ? kind : KK_FFT_X_INV, s, RB + CB);
    const int nblk = N * N / RowTile<R, N>::ROWS;
    k_fft_x_c2r<R, N><<<x_grid(nblk), RowTile<R, N>::THREADS, smem_x(), s>>>(in, out, P, nblk);
  }
  // column pass over all N planes through the TMA pipeline (err != null) or
  // the plain tile kernel
  template <bool ZAXIS>
  static cudaError_t cols_tma(C* d, int P, bool inv, cudaStream_t s, int* err) {
    CUtensorMap map;
    if (!make_cols_map(&map, d, N, P, TT::W, TT::BOXR, ZAXIS, sizeof(R) == 8)) return cudaErrorInvalidValue;
    const int ntx = (N / 2 + 1 + TT::W - 1) / TT::W, tiles = ntx * N;
    if (inv)
      k_fft_cols_tma<R, N, true, ZAXIS><<<tma_grid(tiles), TT::THREADS, TT::SMEM, s>>>(map, map, ntx, tiles, err, R(0));
    else
      k_fft_cols_tma<R, N, false, ZAXIS><<<tma_grid(tiles), TT::THREADS, TT::SMEM, s>>>(map, map, ntx, tiles, err, R(0));
    return cudaSuccess;
  }
  // inverse y pass of a shared x,y gradient spectrum G (in place): d <- i k_x IFFT_y(G),
  // d2 <- IFFT_y(i k_y G)
  static cudaError_t y_dual(C* d, C* d2, int P, double kf, cudaStream_t s, Prof* pf, int kind, int* err) {
    ProfScope ps(pf, kind >= 0 ? kind : KK_FFT_Y_INV, s, 3 * CB);
    CUtensorMap map, map2;
    if (!make_cols_map(&map, d, N, P, TT::W, TT::BOXR, false, sizeof(R) == 8) ||
        !make_cols_map(&map2, d2, N, P, TT::W, TT::BOXR, false, sizeof(R) == 8))
      return cudaErrorInvalidValue;
    const int ntx = (N / 2 + 1 + TT::W - 1) / TT::W, tiles = ntx * N;
    static std::once_flag once[kMaxDevices];
    static int slot_v[kMaxDevices];
    const int slots =
        device_slots(once, slot_v, k_fft_cols_tma<R, N, true, false, true>, TT::THREADS, (size_t)TT::SMEM_DUAL);
    k_fft_cols_tma<R, N, true, false, true><<<std::min(tiles, slots), TT::THREADS, TT::SMEM_DUAL, s>>>(
        map, map2, ntx, tiles, err, (R)kf);
    return cudaSuccess;
  }
  // y pass: planes = z (stride N*P), rows = y (stride P)
  static cudaError_t y(C* d, int P, bool inv, cudaStream_t s, Prof* pf, int kind, int* err) {
    ProfScope ps(pf, kind >= 0 ? kind : (inv ? KK_FFT_Y_INV : KK_FFT_Y_FWD), s, 2 * CB);
    if (err) return cols_tma<false>(d, P, inv, s, err);
    dim3 g(ntiles(), N);
    if (inv) k_fft_cols<R, N, true><<<g, ColTile<R, N>::THREADS, smem_cols(), s>>>(d, (long long)N * P, P, N / 2 + 1);
    else k_fft_cols<R, N, false><<<g, ColTile<R, N>::THREADS, smem_cols(), s>>>(d, (long long)N * P, P, N / 2 + 1);
    return cudaSuccess;
  }
  // z pass: planes = y (stride P), rows = z (stride N*P)
  static cudaError_t z(C* d, int P, bool inv, cudaStream_t s, Prof* pf, int kind, int* err) {
    ProfScope ps(pf, kind >= 0 ? kind : KK_FFT_Z_FWD, s, 2 * CB);
    if (err) return cols_tma<true>(d, P, inv, s, err);
    dim3 g(ntiles(), N);
    if (inv) k_fft_cols<R, N, true><<<g, ColTile<R, N>::THREADS, smem_cols(), s>>>(d, P, (long long)N * P, N / 2 + 1);
    else k_fft_cols<R, N, false><<<g, ColTile<R, N>::THREADS, smem_cols(), s>>>(d, P, (long long)N * P, N / 2 + 1);
    return cudaSuccess;
  }
  // fused z pass.  Force operators with an error word: the TMA pipeline, writing G and F_z
  // (and G_p, S_z) -- the x,y components come from the dual y pass; else the tile kernel.
  static cudaError_t zop(const C* in, const OutPtrs& o, int nout, int P, const SpecParams& sp, cudaStream_t s,
                         Prof* pf, int kind) {
    const bool force = sp.op == OP_FORCE || sp.op == OP_FORCE_PGD;
    if (force && sp.err && (nout == 3 || nout == 6)) {
      using ZT = ZTma<R, N>;
      const int npass = nout == 6 ? 4 : 2;
      ProfScope ps(pf, kind >= 0 ? kind : KK_FFT_Z_OP, s, (1 + npass) * CB);
      CUtensorMap in_map;
      ZOutMaps om;
      const int oi[4] = {0, 2, 3, 5};
      bool ok = make_cols_map(&in_map, const_cast<C*>(in), N, P, ZT::W, ZT::BOXR, true, sizeof(R) == 8);
      for (int q = 0; q < 4 && ok; ++q)
        ok = make_cols_map(&om.m[q], o.p[q < npass ? oi[q] : 0], N, P, ZT::W, ZT::BOXR, true, sizeof(R) == 8);
      if (!ok) return cudaErrorInvalidValue;
      const int ntx = (N / 2 + 1 + ZT::W - 1) / ZT::W, tiles = ntx * N;
      static std::once_flag once[kMaxDevices];
      static int slot_v[kMaxDevices];
      const int slots = device_slots(once, slot_v, k_zpass_op_tma<R, N>, ZT::THREADS, (size_t)ZT::SMEM);
      k_zpass_op_tma<R, N><<<std::min(tiles, slots), ZT::THREADS, ZT::SMEM, s>>>(in_map, om, ntx, tiles, npass, sp,
                                                                                 sp.err);
      return cudaSuccess;
    }
    ProfScope ps(pf, kind >= 0 ? kind : KK_FFT_Z_OP, s, (1 + nout) * CB);
    dim3 g((N / 2 + 1 + ZTile<R, N>::W - 1) / ZTile<R, N>::W, N);
    k_zpass_op<R, N><<<g, ZTile<R, N>::THREADS, smem_z(), s>>>(in, o, nout, P, sp);
    return cudaSuccess;
  }

  // x and y forward passes of real inputs into half spectra (the first stage of a transpose)
  static cudaError_t forward_xy(R* const* real_in, int nin, void* const* ubufs, int P, const SpecParams& sp,
                                cudaStream_t s, Prof* pf) {
    attrs();
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < nin && !e; ++i) {
      C* u = reinterpret_cast<C*>(ubufs[i]);
      x_fwd(real_in[i], u, P, s, pf, KK_ADJ_FFT);
      e = y(u, P, false, s, pf, KK_ADJ_FFT, sp.err);
    }
    return e ? e : cudaGetLastError();
  }

  // x pass of NL lanes of an FP32 mesh interleaved per cell (LANES values per cell) into
  // ubufs[0 .. NL-1], then the y pass of each
  template <int LANES, int NL>
  static cudaError_t forward_xy_il(const R* il, void* const* ubufs, int P, const SpecParams& sp, cudaStream_t s,
                                   Prof* pf) {
    if constexpr (std::is_same<R, float>::value) {
      attrs();
      {
        // the interleaved mesh read, NL half spectra written
        ProfScope ps(pf, KK_ADJ_FFT, s, (double)LANES * RB + (double)NL * CB);
        ILOut o = {};
        for (int q = 0; q < NL; ++q) o.p[q] = reinterpret_cast<float2*>(ubufs[q]);
        k_fft_x_r2c_il<N, LANES, NL><<<(long long)N * N / RowTileIL<N, NL>::ROWS, RowTileIL<N, NL>::THREADS,
                                       RowTileIL<N, NL>::SMEM, s>>>(il, o, P);
      }
      cudaError_t e = cudaSuccess;
      for (int i = 0; i < NL && !e; ++i) e = y(reinterpret_cast<C*>(ubufs[i]), P, false, s, pf, KK_ADJ_FFT, sp.err);
      return e ? e : cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }

  // inputs i < npre are already x,y-transformed in ubufs[i]
  static cudaError_t transpose(R* const* real_in, int nin, int npre, int first, void* const* ubufs, void* cbuf,
                               R* real_out, int P, const SpecParams& sp, cudaStream_t s, Prof* pf) {
    attrs();
    InPtrs ip;
    for (int i = 0; i < 9; ++i) ip.p[i] = i < nin ? ubufs[i] : nullptr;
    cudaError_t e = cudaSuccess;
    for (int i = npre; i < nin && !e; ++i) {
      C* u = reinterpret_cast<C*>(ubufs[i]);
      x_fwd(real_in[i], u, P, s, pf, KK_ADJ_FFT);
      e = y(u, P, false, s, pf, KK_ADJ_FFT, sp.err);
    }
    if (e) return e;
    C* c = reinterpret_cast<C*>(cbuf);
    {
      ProfScope ps(pf, KK_ADJ_FFT, s, (nin + 1) * CB);
      dim3 g((N / 2 + 1 + ZTile<R, N>::W - 1) / ZTile<R, N>::W, N);
      k_zpass_combine<R, N><<<g, ZTile<R, N>::THREADS, smem_z(), s>>>(ip, nin, first, c, P, sp);
    }
    if ((e = y(c, P, true, s, pf, KK_ADJ_FFT, sp.err))) return e;
    x_inv(c, real_out, P, s, pf, KK_ADJ_FFT);
    return cudaGetLastError();
  }

  static cudaError_t r2c(const R* real, void* cplx, int P, cudaStream_t s, Prof* pf, int* err) {
    attrs();
    C* c = reinterpret_cast<C*>(cplx);
    x_fwd(real, c, P, s, pf, -1);
    cudaError_t e = y(c, P, false, s, pf, -1, err);
    if (!e) e = z(c, P, false, s, pf, -1, err);
    return e ? e : cudaGetLastError();
  }

  static cudaError_t apply(const R* real_in, void* cbuf, void* const* ubufs, R* const* real_out, int nout, int P,
                           const SpecParams& sp, cudaStream_t s, Prof* pf, int kind) {
    attrs();
    C* c = reinterpret_cast<C*>(cbuf);
    x_fwd(real_in, c, P, s, pf, kind);
    cudaError_t e = y(c, P, false, s, pf, kind, sp.err);
    if (e) return e;
    OutPtrs o;
    for (int i = 0; i < 9; ++i) o.p[i] = i < nout ? ubufs[i] : nullptr;
    if ((e = zop(c, o, nout, P, sp, s, pf, kind))) return e;
    const bool force = sp.op == OP_FORCE || sp.op == OP_FORCE_PGD;
    if (force && sp.err && (nout == 3 || nout == 6)) {
      // the z pass left G (x,y group) and the z component of each group of three
      for (int g0 = 0; g0 < nout && !e; g0 += 3) {
        e = y_dual(reinterpret_cast<C*>(ubufs[g0]), reinterpret_cast<C*>(ubufs[g0 + 1]), P, sp.kf, s, pf, kind,
                   sp.err);
        if (!e) e = y(reinterpret_cast<C*>(ubufs[g0 + 2]), P, true, s, pf, kind, sp.err);
      }
      for (int i = 0; i < nout && !e; ++i) x_inv(reinterpret_cast<C*>(ubufs[i]), real_out[i], P, s, pf, kind);
      if (e) return e;
    } else {
      for (int i = 0; i < nout; ++i) {
        C* u = reinterpret_cast<C*>(ubufs[i]);
        if ((e = y(u, P, true, s, pf, kind, sp.err))) return e;
        x_inv(u, real_out[i], P, s, pf, kind);
      }
    }
    return cudaGetLastError();
  }
};

#define PM_FFT_DISPATCH(n, EXPR)                       \
  switch (n) {                                         \
    case 32: { using L = Launch<R, 32>; return EXPR; } \
    case 64: { using L = Launch<R, 64>; return EXPR; } \
    case 96: { using L = Launch<R, 96>; return EXPR; } \
    case 128: { using L = Launch<R, 128>; return EXPR; } \
    case 192: { using L = Launch<R, 192>; return EXPR; } \
    case 256: { using L = Launch<R, 256>; return EXPR; } \
    case 512: { using L = Launch<R, 512>; return EXPR; } \
    case 1024: { using L = Launch<R, 1024>; return EXPR; } \
    default: return cudaErrorInvalidValue;             \
  }

}  // namespace

template <typename R>
cudaError_t fft3d_r2c(const R* real, void* cplx, int n, int P, cudaStream_t s, Prof* pf, int* err) {
  PM_FFT_DISPATCH(n, L::r2c(real, cplx, P, s, pf, err));
}

template <typename R>
cudaError_t spectral_apply(const R* real_in, void* cbuf, void* const* ubufs, R* const* real_out, int nout, int n,
                           int P, const SpecParams& sp, cudaStream_t s, Prof* pf, int kind) {
  if (nout < 1 || nout > 9) return cudaErrorInvalidValue;
  PM_FFT_DISPATCH(n, L::apply(real_in, cbuf, ubufs, real_out, nout, P, sp, s, pf, kind));
}

template <typename R>
cudaError_t spectral_transpose(R* const* real_in, int nin, int first, void* const* ubufs, void* cbuf, R* real_out,
                               int n, int P, const SpecParams& sp, cudaStream_t s, Prof* pf) {
  if (nin < 1 || nin > 9) return cudaErrorInvalidValue;
  PM_FFT_DISPATCH(n, L::transpose(real_in, nin, 0, first, ubufs, cbuf, real_out, P, sp, s, pf));
}

template <typename R>
cudaError_t spectral_transpose_pre(R* const* real_in, int nin, int npre, int first, void* const* ubufs, void* cbuf,
                                   R* real_out, int n, int P, const SpecParams& sp, cudaStream_t s, Prof* pf) {
  if (nin < 1 || nin > 9 || npre < 0 || npre > nin) return cudaErrorInvalidValue;
  PM_FFT_DISPATCH(n, L::transpose(real_in, nin, npre, first, ubufs, cbuf, real_out, P, sp, s, pf));
}

template <typename R>
cudaError_t spectral_forward_xy(R* const* real_in, int nin, void* const* ubufs, int n, int P, const SpecParams& sp,
                                cudaStream_t s, Prof* pf) {
  if (nin < 1 || nin > 9) return cudaErrorInvalidValue;
  PM_FFT_DISPATCH(n, L::forward_xy(real_in, nin, ubufs, P, sp, s, pf));
}

template <typename R>
cudaError_t spectral_forward_xy_il(const R* il, int lanes, int nl, void* const* ubufs, int n, int P,
                                   const SpecParams& sp, cudaStream_t s, Prof* pf) {
  if (lanes == 4 && nl == 3) { PM_FFT_DISPATCH(n, (L::template forward_xy_il<4, 3>(il, ubufs, P, sp, s, pf))); }
  if (lanes == 4 && nl == 4) { PM_FFT_DISPATCH(n, (L::template forward_xy_il<4, 4>(il, ubufs, P, sp, s, pf))); }
  if (lanes == 2 && nl == 2) { PM_FFT_DISPATCH(n, (L::template forward_xy_il<2, 2>(il, ubufs, P, sp, s, pf))); }
  return cudaErrorInvalidValue;
}

template cudaError_t spectral_transpose<PM_REAL>(PM_REAL* const*, int, int, void* const*, void*, PM_REAL*, int, int,
                                                  const SpecParams&, cudaStream_t, Prof*);
template cudaError_t spectral_transpose_pre<PM_REAL>(PM_REAL* const*, int, int, int, void* const*, void*, PM_REAL*,
                                                      int, int, const SpecParams&, cudaStream_t, Prof*);
template cudaError_t spectral_forward_xy<PM_REAL>(PM_REAL* const*, int, void* const*, int, int, const SpecParams&,
                                                   cudaStream_t, Prof*);
template cudaError_t spectral_forward_xy_il<PM_REAL>(const PM_REAL*, int, int, void* const*, int, int,
                                                      const SpecParams&, cudaStream_t, Prof*);
template cudaError_t fft3d_r2c<PM_REAL>(const PM_REAL*, void*, int, int, cudaStream_t, Prof*, int*);
template cudaError_t spectral_apply<PM_REAL>(const PM_REAL*, void*, void* const*, PM_REAL* const*, int, int, int,
                                              const SpecParams&, cudaStream_t, Prof*, int);

}  // namespace pmlens
