// Device code shared by the single-problem and batched SpMM kernels.
#pragma once

#include <cuda_bf16.h>

#include "device.h"
#include "dot.cuh"

namespace amgsym {

template <typename T>
struct AccOf {
  using type = float;
};
template <>
struct AccOf<double> {
  using type = double;
};

template <typename T>
__device__ __forceinline__ float to_f(T v) {
  return (float)v;
}
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

template <typename A, typename T>
__device__ __forceinline__ A cvt(T v) {
  return (A)v;
}
template <>
__device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <>
__device__ __forceinline__ double cvt<double, __nv_bfloat16>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}

// Vector of N consecutive T, aligned to its size up to 32 bytes (a 32-byte
// vector is one 256-bit access where the hardware has it, else two 16-byte ones).
template <typename T, int N>
struct alignas(sizeof(T) * N <= 32 ? sizeof(T) * N : 32) Vec {
  T v[N];
};

template <typename T, int N>
__device__ __forceinline__ Vec<T, N> ldv(const T* p) {
  return *reinterpret_cast<const Vec<T, N>*>(p);
}
// 32-byte vectors as one 256-bit load (ld.global.v8.f32 / .v4.f64, sm_100 and
// later): one request per warp instruction instead of two 128-bit ones.
template <>
__device__ __forceinline__ Vec<float, 8> ldv<float, 8>(const float* p) {
  Vec<float, 8> r;
  asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]), "=f"(r.v[5]), "=f"(r.v[6]),
                 "=f"(r.v[7])
               : "l"(p));
  return r;
}
template <>
__device__ __forceinline__ Vec<double, 4> ldv<double, 4>(const double* p) {
  Vec<double, 4> r;
  asm volatile("ld.global.v4.f64 {%0, %1, %2, %3}, [%4];"
               : "=d"(r.v[0]), "=d"(r.v[1]), "=d"(r.v[2]), "=d"(r.v[3])
               : "l"(p));
  return r;
}
// The same load through L2 only (ld.global.cg): coherent with what other
// blocks of the same launch wrote before a grid barrier (the persistent
// coarse-cycle kernel), unlike the read-only data path.
template <typename T, int N>
__device__ __forceinline__ Vec<T, N> ldv_cg(const T* p) {
  Vec<T, N> r;
  constexpr int B = (int)sizeof(T) * N;
  if constexpr (B % 16 == 0) {
#pragma unroll
    for (int i = 0; i < B / 16; ++i) reinterpret_cast<uint4*>(&r)[i] = __ldcg(reinterpret_cast<const uint4*>(p) + i);
  } else if constexpr (B % 8 == 0) {
#pragma unroll
    for (int i = 0; i < B / 8; ++i) reinterpret_cast<uint2*>(&r)[i] = __ldcg(reinterpret_cast<const uint2*>(p) + i);
  } else {
    static_assert(B % 4 == 0, "vector of 4-byte multiples");
#pragma unroll
    for (int i = 0; i < B / 4; ++i)
      reinterpret_cast<unsigned*>(&r)[i] = __ldcg(reinterpret_cast<const unsigned*>(p) + i);
  }
  return r;
}
template <typename T, int N, bool COH>
__device__ __forceinline__ Vec<T, N> ldx(const T* p) {
  if constexpr (COH)
    return ldv_cg<T, N>(p);
  else
    return ldv<T, N>(p);
}
template <typename T, int N>
__device__ __forceinline__ void stv(T* p, const Vec<T, N>& v) {
  *reinterpret_cast<Vec<T, N>*>(p) = v;
}

// The compute type: FP64 if either operand is FP64, else FP32.
template <typename MT, typename XT>
struct ComputeOf {
  using type = float;
};
template <typename XT>
struct ComputeOf<double, XT> {
  using type = double;
};
template <typename MT>
struct ComputeOf<MT, double> {
  using type = double;
};
template <>
struct ComputeOf<double, double> {
  using type = double;
};

// The entries of one row in the diagonal-offset form: every value load and
// gather of a batch of diagonals issued before its FMAs (no dependent index
// loads: the columns are row + offset); one batch holds all diagonals with
// 16-byte column vectors and four with 32-byte ones (registers).  The sum
// runs over the diagonals in ascending offset, i.e. column, order -- the
// order of the CSR loop -- and skips columns outside [0, rows); padded
// positions inside hold 0 and add fma(0, x, acc) = acc.
template <typename MT, typename XT, typename CT, int CPT, bool COH>
__device__ __forceinline__ void dia_row(const SpmmArgs& a, int row, int c0, CT (&acc)[CPT]) {
  const MT* __restrict__ dv = static_cast<const MT*>(a.dval);
  const XT* __restrict__ X = static_cast<const XT*>(a.X);
  const int64_t n = a.dstride;
  constexpr int UB = CPT * sizeof(XT) >= 32 ? 4 : kMaxDiag;
#pragma unroll
  for (int d0 = 0; d0 < kMaxDiag; d0 += UB) {
    if (d0 < a.ndiag) {
      CT m[UB];
      Vec<XT, CPT> x[UB];
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int d = d0 + u;
        const int j = row + a.doff[d];
        const bool ok = d < a.ndiag && (unsigned)j < (unsigned)a.rows;
        m[u] = ok ? cvt<CT>(dv[(int64_t)a.dsrc[d] * n + row + a.dshift[d]]) : (CT)0;
        if (ok) {
          x[u] = ldx<XT, CPT, COH>(X + (int64_t)j * a.C + c0);
        } else {
#pragma unroll
          for (int q = 0; q < CPT; ++q) x[u].v[q] = (XT)0;
        }
      }
#pragma unroll
      for (int u = 0; u < UB; ++u) {
#pragma unroll
        for (int q = 0; q < CPT; ++q) acc[q] = fma(m[u], (CT)x[u].v[q], acc[q]);
      }
    }
  }
}

// The CSR entries kb + e, kb + e + KL, ... < ke of one row, U per step,
// predicated: all index/value loads first, then all gathers, so a row of up
// to U * KL entries costs one round trip and a 7-point row (U = 4) two, with
// every gather of a step in flight at once.
template <typename MT, typename XT, typename CT, int CPT, int KL, bool COH>
__device__ __forceinline__ void csr_row(const SpmmArgs& a, int kb, int ke, int e, int c0, CT (&acc)[CPT]) {
  const MT* __restrict__ val = static_cast<const MT*>(a.val);
  const XT* __restrict__ X = static_cast<const XT*>(a.X);
  const int32_t* __restrict__ idx = a.idx;
  const int C = a.C;
  constexpr int U = CPT >= 8 ? 2 : 4;
  for (int k = kb + e; k < ke; k += U * KL) {
    int j[U];
    CT m[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = k + u * KL < ke;
      j[u] = ok ? __ldg(idx + k + u * KL) : 0;
      m[u] = ok ? cvt<CT>(val[k + u * KL]) : (CT)0;
    }
    Vec<XT, CPT> x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k + u * KL < ke) {
        x[u] = ldx<XT, CPT, COH>(X + (int64_t)j[u] * C + c0);
      } else {
#pragma unroll
        for (int q = 0; q < CPT; ++q) x[u].v[q] = (XT)0;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int q = 0; q < CPT; ++q) acc[q] = fma(m[u], (CT)x[u].v[q], acc[q]);
    }
  }
}

// The entries kb + e, kb + e + KL, ... < ke of one row of a halo-staged
// matrix: the same batches, masking and fma sequence as csr_row (so the same
// sums), with 16-bit column indices into the tile's halo and the gathered
// rows read from shared memory (xs: [halo][C], staged by the caller).
template <typename MT, typename XT, typename CT, int CPT, int KL>
__device__ __forceinline__ void halo_row(const SpmmArgs& a, const XT* xs, int kb, int ke, int e, int c0,
                                         CT (&acc)[CPT]) {
  const MT* __restrict__ val = static_cast<const MT*>(a.val);
  const uint16_t* __restrict__ li = a.lidx;
  const int C = a.C;
  // 8 entries per lane per batch (one global round trip for the index and
  // value loads of rows up to 8 * KL entries); each gathered row comes from
  // shared memory right before its fmas.  The fma sequence of every lane is
  // that of csr_row (entries in order, a masked entry adds fma(0, 0, acc)).
  constexpr int U = 8;
  for (int k = kb + e; k < ke; k += U * KL) {
    int j[U];
    CT m[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = k + u * KL < ke;
      j[u] = ok ? (int)__ldg(li + k + u * KL) : 0;
      m[u] = ok ? cvt<CT>(val[k + u * KL]) : (CT)0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      Vec<XT, CPT> x;
      if (k + u * KL < ke) {
        x = *reinterpret_cast<const Vec<XT, CPT>*>(xs + j[u] * C + c0);
      } else {
#pragma unroll
        for (int q = 0; q < CPT; ++q) x.v[q] = (XT)0;
      }
#pragma unroll
      for (int q = 0; q < CPT; ++q) acc[q] = fma(m[u], (CT)x.v[q], acc[q]);
    }
  }
}

// The interface couplings of flagged row number f (A_out,i of eq.
// "hL_splitting"; one value per block column).
template <typename XT, typename CT, int CPT, bool COH>
__device__ __forceinline__ void iface_row(const SpmmArgs& a, int f, int c0, CT (&acc)[CPT]) {
  const CT* __restrict__ iv = static_cast<const CT*>(a.ival);
  const XT* __restrict__ X = static_cast<const XT*>(a.X);
  for (int ee = __ldg(a.iptr + f); ee < __ldg(a.iptr + f + 1); ++ee) {
    const int j = __ldg(a.icol + ee);
    const Vec<XT, CPT> xv = ldx<XT, CPT, COH>(X + (int64_t)j * a.C + c0);
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const int blk = (c0 + q) % a.nb;
      acc[q] = fma(iv[(int64_t)ee * a.nb + blk], (CT)xv.v[q], acc[q]);
    }
  }
}

// Number of flagged rows before `row` (row <= rows).
__device__ __forceinline__ int flag_index(const SpmmArgs& a, int row) {
  if (row >= a.rows) return a.nflag;
  const uint32_t wd = __ldg(a.imask + (row >> 5));
  return __ldg(a.iprefix + (row >> 5)) + __popc(wd & ((1u << (row & 31)) - 1u));
}

// Epilogue of one row (entry lane 0): Y = alpha acc + beta Z, the optional dot.
template <typename XT, typename OT, typename CT, typename DT, int CPT, bool HAS_DOT, bool COH>
__device__ __forceinline__ void row_epilogue(const SpmmArgs& a, int row, int c0, CT (&acc)[CPT],
                                             const Vec<XT, CPT>& zpre, bool use_zpre, const Vec<XT, CPT>& wpre,
                                             bool use_wpre, DT (&dpart)[CPT]) {
  const int C = a.C;
  const CT alpha = (CT)a.alpha, beta = (CT)a.beta;
  // Y may alias Z (in-place update z += ...); each row reads Z before writing Y.
  OT* Y = static_cast<OT*>(a.Y);
  Vec<OT, CPT> out;
  if (a.beta != 0.0) {
    // the epilogue operand as loaded early by the caller (use_zpre), else now;
    // passed by value so that it stays in registers
    const Vec<XT, CPT> zv = use_zpre ? zpre : ldx<XT, CPT, COH>(static_cast<const XT*>(a.Z) + (int64_t)row * C + c0);
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const CT y = fma(alpha, acc[q], beta * (CT)zv.v[q]);
      out.v[q] = (OT)y;
      acc[q] = y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const CT y = alpha * acc[q];
      out.v[q] = (OT)y;
      acc[q] = y;
    }
  }
  if (a.jmode == 1) {
    // presmoothing of the next level from zero: Y2 = jd o Y, the arithmetic
    // of the stand-alone diagonal step (one product of the stored values)
    const XT d = static_cast<const XT*>(a.jd)[row];
    Vec<OT, CPT> o2;
#pragma unroll
    for (int q = 0; q < CPT; ++q) o2.v[q] = (OT)(d * (XT)out.v[q]);
    stv<OT, CPT>(static_cast<OT*>(a.Y2) + (int64_t)row * C + c0, o2);
  } else if (a.jmode == 2) {
    // postsmoothing: X + jd o r with r the stored residual value
    const XT d = static_cast<const XT*>(a.jd)[row];
    const Vec<XT, CPT> xr = ldx<XT, CPT, COH>(static_cast<const XT*>(a.X) + (int64_t)row * C + c0);
#pragma unroll
    for (int q = 0; q < CPT; ++q) out.v[q] = (OT)fma(d, (XT)out.v[q], xr.v[q]);
  }
  stv<OT, CPT>(Y + (int64_t)row * C + c0, out);
  if (HAS_DOT) {
    if (a.dot.mode == DOT_WY) {
      // the dot partner as loaded early by the caller (use_wpre), else now
      const Vec<XT, CPT> wv =
          use_wpre ? wpre : ldx<XT, CPT, COH>(static_cast<const XT*>(a.dot.W) + (int64_t)row * C + c0);
#pragma unroll
      for (int q = 0; q < CPT; ++q) dpart[q] = fma((DT)wv.v[q], (DT)acc[q], dpart[q]);
    } else {
#pragma unroll
      for (int q = 0; q < CPT; ++q) dpart[q] = fma((DT)acc[q], (DT)acc[q], dpart[q]);
    }
  }
}

// Rows [first_slot * rows_pb + k * slot_step * rows_pb, ...) below row_end
// of one SpMM, for the whole block; this thread's dot partial (entry lane 0
// only) is added to dpart.  Thread layout: a row is served by S = TPC * KL
// threads: TPC column threads (each owning CPT consecutive columns, TPC =
// C / CPT) times KL entry lanes (lane e takes the row's entries e, e + KL,
// ...).  The KL partial sums are combined with warp shuffles (S divides 32
// when KL > 1), and entry lane 0 runs the epilogue.  KL > 1 keeps several
// gathers of one row in flight (the ptr -> idx -> X latency chain) and spreads
// the long rows of the coarse levels over many lanes.  DIA: the matrix is in
// the diagonal-offset form (one lane per row, no row pointers).  COH: vector
// operands are loaded through L2 only (written earlier in the same launch).
//
// Interface rows (HAS_IFACE) take a second pass: the main pass computes
// every row but stores none of the flagged ones, so no row waits on the
// flag -> prefix -> pointer -> coupling chain; then the flagged rows (about
// 2 % of them at 256^3) are recomputed with their couplings, from the
// compact list of flagged rows.  whole: the block's share of the whole
// matrix (the flagged rows slotted like the rows); otherwise the block owns
// rows [first_slot * rows_pb, row_end) alone and takes their flagged rows.
// A flagged row's sum is the same in both designs: its entries, then its
// couplings (entry lane 0), then the lane combination.
template <typename MT, typename XT, typename OT, int CPT, int KL, bool HAS_DOT, bool HAS_IFACE, bool DIA = false,
          bool COH = false>
__device__ __forceinline__ void spmm_tile(const SpmmArgs& a, int first_slot, int slot_step, int row_end,
                                          typename AccOf<XT>::type (&dpart)[CPT], bool whole = true) {
  static_assert(!DIA || KL == 1, "the diagonal-offset form runs one entry lane per row");
  using CT = typename ComputeOf<MT, XT>::type;
  using DT = typename AccOf<XT>::type;  // per-thread dot partial type
  // Early epilogue-operand loads, issued with the row's matrix and X loads so
  // that the epilogue adds no dependent round trip: Z (beta != 0) in the CSR
  // variants launched at 6 blocks per SM, Z and the dot partner W in the
  // diagonal-form dot variants (3 blocks per SM, registers to spare).
  constexpr bool ZPF = (HAS_DOT || HAS_IFACE) && !DIA;
  constexpr bool DPF = HAS_DOT && DIA;
  constexpr bool PTR_PF = ZPF && !DIA;
  const int C = a.C;
  const int TPC = C / CPT;
  const int S = TPC * KL;
  const int rows_pb = kBlock / S;
  const int g = threadIdx.x / S;
  const int w = threadIdx.x - g * S;
  const int e = KL > 1 ? w / TPC : 0;
  const int c0 = (w - e * TPC) * CPT;
  const bool slot_ok = g < rows_pb;
  const XT* Z = static_cast<const XT*>(a.Z);
  const int32_t* __restrict__ ptr = a.ptr;
  auto lanes = [&](CT (&acc)[CPT]) {
    if (KL > 1) {
#pragma unroll
      for (int off = KL / 2; off >= 1; off >>= 1) {
#pragma unroll
        for (int q = 0; q < CPT; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off * TPC);
      }
    }
  };

  // The trip count is block-uniform (the shuffles need every lane of the warp).
  // In the variants with registers to spare (ZPF), the row pointers of a
  // thread's next row are loaded one iteration ahead, which takes one
  // dependent load off each row's chain.
  const int step_rows = slot_step * rows_pb;
  int kb_next = 0, ke_next = 0;
  if (PTR_PF) {
    const int row0 = first_slot * rows_pb + g;
    if (slot_ok && row0 < row_end) {
      kb_next = __ldg(ptr + row0);
      ke_next = __ldg(ptr + row0 + 1);
    }
  }
  for (int base = first_slot * rows_pb; base < row_end; base += step_rows) {
    const int row = base + g;
    const bool live = slot_ok && row < row_end;
    CT acc[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) acc[q] = (CT)0;
    Vec<XT, CPT> zpre, wpre;
    int kb = kb_next, ke = ke_next;
    if (PTR_PF) {
      if (slot_ok && row + step_rows < row_end) {
        kb_next = __ldg(ptr + row + step_rows);
        ke_next = __ldg(ptr + row + step_rows + 1);
      }
    } else if (!DIA && live) {
      kb = __ldg(ptr + row);
      ke = __ldg(ptr + row + 1);
    }
    bool flagged = false;
    if (live) {
      // interface flag word and epilogue operand loaded with the row pointers,
      // off the critical path of the gathers
      const uint32_t iface_word = (HAS_IFACE && e == 0) ? __ldg(a.imask + (row >> 5)) : 0u;
      if ((ZPF || DPF) && e == 0 && a.beta != 0.0) zpre = ldx<XT, CPT, COH>(Z + (int64_t)row * C + c0);
      if (DPF && e == 0 && a.dot.mode == DOT_WY)
        wpre = ldx<XT, CPT, COH>(static_cast<const XT*>(a.dot.W) + (int64_t)row * C + c0);
      if (DIA)
        dia_row<MT, XT, CT, CPT, COH>(a, row, c0, acc);
      else
        csr_row<MT, XT, CT, CPT, KL, COH>(a, kb, ke, e, c0, acc);
      flagged = HAS_IFACE && (iface_word >> (row & 31)) & 1u;
    }
    lanes(acc);
    if (live && e == 0 && !flagged)
      row_epilogue<XT, OT, CT, DT, CPT, HAS_DOT, COH>(a, row, c0, acc, zpre, (ZPF || DPF) && a.beta != 0.0, wpre,
                                                      DPF && a.dot.mode == DOT_WY, dpart);
  }
  if (HAS_IFACE) {
    // the flagged rows, with their couplings
    const int f_begin = whole ? 0 : flag_index(a, first_slot * rows_pb);
    const int f_end = whole ? a.nflag : flag_index(a, row_end);
    const int fs0 = whole ? first_slot : 0, fstep = whole ? slot_step : 1;
    for (int fb = f_begin + fs0 * rows_pb; fb < f_end; fb += fstep * rows_pb) {
      const int f = fb + g;
      const bool live = slot_ok && f < f_end;
      const int row = live ? __ldg(a.irows + f) : 0;
      CT acc[CPT];
#pragma unroll
      for (int q = 0; q < CPT; ++q) acc[q] = (CT)0;
      if (live) {
        if (DIA) {
          dia_row<MT, XT, CT, CPT, COH>(a, row, c0, acc);
        } else {
          csr_row<MT, XT, CT, CPT, KL, COH>(a, __ldg(ptr + row), __ldg(ptr + row + 1), e, c0, acc);
        }
        if (e == 0) iface_row<XT, CT, CPT, COH>(a, f, c0, acc);
      }
      lanes(acc);
      if (live && e == 0)
        row_epilogue<XT, OT, CT, DT, CPT, HAS_DOT, COH>(a, row, c0, acc, Vec<XT, CPT>{}, false, Vec<XT, CPT>{}, false,
                                                        dpart);
    }
  }
}

// The thread's place in the tile layout (see spmm_tile).
struct TileLayout {
  int S, rows_pb, g, e, c0;
  bool slot_ok;
};

template <int CPT, int KL>
__device__ __forceinline__ TileLayout tile_layout(int C) {
  TileLayout t;
  const int TPC = C / CPT;
  t.S = TPC * KL;
  t.rows_pb = kBlock / t.S;
  t.g = threadIdx.x / t.S;
  const int w = threadIdx.x - t.g * t.S;
  t.e = KL > 1 ? w / TPC : 0;
  t.c0 = (w - t.e * TPC) * CPT;
  t.slot_ok = t.g < t.rows_pb;
  return t;
}

}  // namespace amgsym
