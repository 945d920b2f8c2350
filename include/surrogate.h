/*
 * surrogate.h -- C ABI of the kernels of the learned near-field surrogate
 * (libfdtd_gb300.so).
 *
 * The paper has no counterpart to any call here.  The surrogate is a small
 * network trained on traces that the FDTD path of fdtd.h produces; FDTD stays
 * the reference and the fallback.  It learns the field response G(r, dz, t)
 * of one bin of the shower's longitudinal charge profile (an MLP from the
 * antenna's radius and axial offset to a waveform) and sums it over the bins
 * (the traces are linear in the profile, and a uniform medium makes the
 * response depend on the offset between antenna and bin only: the learned
 * counterpart of the Green's function superposition of Sec. II).  These calls
 * are the forward and backward kernels and the optimiser step; the 1D
 * convolutions are general-purpose kernels of the same family.  The lattice
 * model (sur_lattice_*, at the end) replaces the MLP by a learned response
 * table on the grid's own lattice, where the shift invariance is exact.
 *
 * Conventions
 *   - All tensors are device buffers owned by the caller; the calls allocate
 *     nothing and run asynchronously on `stream` (a cudaStream_t, NULL = the
 *     default stream).
 *   - bf16 buffers hold IEEE bfloat16 values (2 bytes); f32 buffers float.
 *   - Activations are row-major [batch][features] or [batch][channel][length].
 *   - Return: FDTD_OK (0), FDTD_ERR_ARG (-1) on a null pointer or a bad size
 *     (detected before any launch), FDTD_ERR_CUDA (-5) if a launch fails.
 */
#ifndef SURROGATE_GB300_H
#define SURROGATE_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Y = op(A) op(B)^T on the tensor cores: bf16 operands, f32 accumulation.
 *   op(A) is M x K: A(m,k) = A[m*lda + k] if a_kmajor, else A[k*lda + m];
 *   op(B) is N x K: B(n,k) = B[n*ldb + k] if b_kmajor, else B[k*ldb + n].
 *   Y[m*ldy + n] (f32) = (accumulate ? Y : 0) + sum_k A(m,k) B(n,k)
 *                        + (bias ? bias[n] : 0), then max(., 0) if relu.
 *   Yb (bf16, may be NULL) receives a rounded copy of Y with the same ldy.
 * M, N, K >= 1.
 */
int sur_gemm_bf16(const void *A, int lda, int a_kmajor, const void *B, int ldb, int b_kmajor, float *Y, int ldy,
                  void *Yb, int M, int N, int K, const float *bias, int relu, int accumulate, void *stream);

/*
 * The kernels behind sur_gemm_bf16.  With both operands K-major, lda and ldb
 * multiples of 8 and A, B 16-byte aligned, the product runs on the
 * fifth-generation tensor cores (tcgen05.mma, accumulator in tensor memory,
 * operands staged by TMA, 128 x 128 output tiles); any other layout on the
 * warp-level mma.sync kernel.  sur_gemm_set_path(p) selects for later calls
 * (process-wide): 0 that automatic choice (the default), 1 mma.sync always,
 * 2 tcgen05 with 128-byte swizzled operand slices only, 3 tcgen05 with
 * unswizzled core-matrix slices only (K a multiple of 8); with 2 or 3 a
 * product the tcgen05 kernel cannot take returns FDTD_ERR_ARG.
 * sur_gemm_tc_launches: launches of the tcgen05 kernel so far.
 * sur_gemm_tc_failed: synchronises the device and returns 1 if a bounded
 * pipeline wait of the tcgen05 kernel gave up since the last call (that
 * CTA's outputs were not written), else 0; FDTD_ERR_CUDA on a CUDA error.
 */
int sur_gemm_set_path(int path);
long long sur_gemm_tc_launches(void);
int sur_gemm_tc_failed(void);

/*
 * batch products on the tcgen05 kernel in one launch:
 *   Y[b][m*ldy + n] = alpha * (row_scale ? row_scale[m] : 1) * sum_k A_b(m,k) B_b(n,k),
 *   A_b(m,k) = A[b*sa + m*lda + k], B_b(n,k) = B[b*sb + n*ldb + k] (bf16, both
 *   K-major; sa or sb = 0: one operand shared by the batch), Y_b at Y + b*sy
 *   (f32; sy >= M*ldy when batch > 1), row_scale f32 [M] or NULL.
 * lda, ldb, sa, sb multiples of 8 and A, B 16-byte aligned; 1 <= batch <=
 * 65535.  FDTD_ERR_ARG otherwise, and while sur_gemm_set_path has selected
 * mma.sync (1) or the unswizzled tcgen05 layout (3).
 */
int sur_gemm_bf16_batched(const void *A, int lda, long long sa, const void *B, int ldb, long long sb, float *Y, int ldy,
                          long long sy, int M, int N, int K, int batch, const float *row_scale, float alpha,
                          void *stream);

/*
 * 1D convolution, f32 activations, bf16 weights, f32 accumulation:
 *   y[b][o][l] = bias[o] + sum_{c,t} w[o][c][t] x[b][c][l*stride + t - pad]
 *   (x read as 0 outside 0..lin-1), then max(., 0) if relu.
 * x: [B][cin][lin] with batch stride xs (floats; >= cin*lin);
 * y: [B][cout][lout], lout = (lin + 2 pad - k) / stride + 1.
 */
int sur_conv1d_fwd(const float *x, int xs, const void *w, const float *bias, float *y, int B, int cin, int lin,
                   int cout, int k, int stride, int pad, int relu, void *stream);

/*
 * Backward of sur_conv1d_fwd with relu = 1.  y is the forward output, dy the
 * gradient with respect to y ([B][cout][lout], batch stride dys).  Writes
 * dw[o][c][t] (f32) and db[o] (f32), overwriting them, and, if dx is not
 * NULL, dx[b][c][i] ([B][cin][lin], batch stride lin*cin).
 */
int sur_conv1d_bwd(const float *x, int xs, const void *w, const float *y, const float *dy, int dys, float *dx,
                   float *dw, float *db, int B, int cin, int lin, int cout, int k, int stride, int pad,
                   void *stream);

/* dz[i] = dy[i] (y[i] > 0), i < n; dzb (bf16, may be NULL) a rounded copy. */
int sur_relu_bwd(const float *y, const float *dy, float *dz, void *dzb, long long n, void *stream);

/* db[n] = sum_m dz[m*ldz + n] (overwrites), n < N, m < M. */
int sur_bias_grad(const float *dz, int ldz, int M, int N, float *db, void *stream);

/* y[i] = bf16(x[i]), i < n. */
int sur_cast_bf16(const float *x, void *y, long long n, void *stream);

/*
 * out[b][0:na] = bf16(a[b][0:na]), out[b][na:na+nc] = bf16(c[b][0:nc]),
 * b < B; a has batch stride na, c batch stride nc, out batch stride na + nc.
 */
int sur_concat_bf16(const float *a, int na, const float *c, int nc, void *out, int B, void *stream);

/*
 * Mean squared error over n elements and its gradient:
 *   dy[i] = 2 (y[i] - t[i]) / n;  loss[0] (f32, device) = sum (y - t)^2 / n
 * (loss may be NULL).
 */
int sur_mse(const float *y, const float *t, long long n, float *dy, float *loss, void *stream);

/*
 * Adam step t >= 1 on n parameters (f32 master copy w, moments m and v):
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps);
 *   wb (bf16, may be NULL) = bf16(w).
 */
int sur_adam(float *w, void *wb, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
             float eps, int t, void *stream);

/*
 * Input scaling: s[b] = max_i |q[b][i]|, qn[b][i] = q[b][i] / s[b] (0 when
 * s[b] = 0), b < B, i < n.  The traces are linear in the profile (the field
 * equations are linear in the current), so the network sees unit-peak
 * profiles and its output is multiplied back by s[b] (sur_scale_rows).
 */
int sur_normalize_rows(const float *q, int B, int n, float *qn, float *s, void *stream);

/*
 * Antenna features, out[b][0..63] (f32) from rz[b] = (r, z) in metres:
 *   u = (r - r0)/rs, v = (z - z0)/zs;  out[0] = u, out[1] = v,
 *   out[2+4(f-1) .. 5+4(f-1)] = sin(f pi u), cos(f pi u), sin(f pi v), cos(f pi v)
 *   for f = 1..15;  out[62] = out[63] = 0.
 */
int sur_antenna_features(const float *rz, int B, float r0, float rs, float z0, float zs, float *out, void *stream);

/* y[b][i] *= c s[b] (invert = 0) or c / s[b] (invert = 1; 0 where s[b] = 0),
   b < B, i < n. */
int sur_scale_rows(float *y, int B, int n, const float *s, float c, int invert, void *stream);

/*
 * Antenna-bin pairs: out[b*K + k] = (rz[b][0], rz[b][1] - z0 - k dz), the
 * antenna's radius and its axial offset from profile bin k (metres), b < B,
 * k < K.
 */
int sur_pairs(const float *rz, int B, int K, float z0, float dz, float *out, void *stream);

/*
 * Superposition of the bins' responses along the shower, each in retarded
 * time (a 1D transposed convolution with a kernel per antenna and bin):
 *   R = |(r_b, dz_bk)| with dz_bk = rz[b][1] - z0 - k dz (metres),
 *   c = shift k + R / cps  (cps: metres the wave covers per sample),
 *   ci = floor(c), f = c - ci,
 *   out[b][i] = sum_k qn[b][k] (1/R) ((1 - f) G[b*K + k][i - ci + J0]
 *                                    + f G[b*K + k][i - ci - 1 + J0])
 *   with G entries outside 0..Tg-1 read as zero, i < T.
 * G: [B*K][Tg] f32 (index J0 is the direct arrival of the bin's field);
 * qn: [B][K]; rz: [B][2]; out: [B][T] (overwritten).  R is floored at dz/2.
 */
int sur_assemble(const float *G, const float *qn, const float *rz, int B, int K, int Tg, int shift, int T, float z0,
                 float dz, float cps, int J0, float *out, void *stream);

/*
 * Its gradient with respect to G (the exact transpose):
 *   dG[b*K + k][j] = qn[b][k] (1/R) ((1 - f) dout[b][j + ci - J0]
 *                                    + f dout[b][j + ci + 1 - J0])
 * (dout read as zero outside 0..T-1), j < Tg; dGb (bf16, may be NULL) a
 * rounded copy.
 */
int sur_assemble_bwd(const float *dout, const float *qn, const float *rz, int B, int K, int Tg, int shift, int T,
                     float z0, float dz, float cps, int J0, float *dG, void *dGb, void *stream);

/*
 * Lattice surrogate.  With the shower moving half a cell per step (c dt =
 * dx/2) and profile bins of 2S steps (S trace samples of two steps each, S
 * cells), the field of bin k at an antenna is the field of bin 0 at the
 * antenna moved S k cells back along z, S k samples earlier: the scheme and
 * the charge-conserving deposit commute with that translation of the grid's
 * lattice (Sec. III.A, III.B).  A trace is linear in the profile.  So, for
 * antennas on the lattice of radial class ir (a node distance from the axis
 * in the plane phi = 0) and axial index m (the antenna at the start of bin m),
 *   y[b][t] = sum_k q[b][k] G[ir][m - k + moff][t - S k + J]
 *                                   (terms with 0 <= t - S k + J < T),
 * where G[ir][d][tau] (NR x D x T, bf16) is the learned response of one bin
 * at lattice offset d - moff and J >= 0 lead samples (with the profile
 * interpolated linearly between bins, bin k's charge starts to move when the
 * shower passes bin k-1: J = S).  The weights of an antenna form a K x T
 * matrix, W[k][t] = G[ir][m - k + moff][t - S k + J], so a batch of profiles at one
 * antenna is a tensor-core GEMM (sur_lattice_weights, then sur_gemm_bf16).
 *   G: bf16 [NR][D][T];  q: f32 [B][K] (K <= 1024);  ant: int [B][2] = (ir, m);
 *   y: f32 [B][T] (overwritten);  dG: f32 [NR][D][T] (accumulated: clear it
 *   first);  offsets outside 0..D-1 and classes outside 0..NR-1 contribute 0.
 * sur_lattice_fwd:  y as above (f32 accumulation) from the bf16 table G, plus
 *                   a second bf16 table Glo of the remainders if not NULL
 *                   (G + Glo carries about 16 significant bits, see
 *                   sur_split_bf16).
 * sur_lattice_fwd_f32: the same from an f32 table (the training master).
 * sur_lattice_bwd:  dG[ir][m - k + moff][tau] += q[b][k] dy[b][tau + S k - J]
 *                   (the exact transpose of the forward map, atomic adds).
 * sur_lattice_weights: W (bf16 [A][K][T]) of A antennas ant[A][2].
 * B, A <= 65535.
 */
int sur_lattice_fwd(const void *G, const void *Glo, const float *q, const int *ant, int B, int K, int NR, int D,
                    int T, int S, int J, int moff, float *y, void *stream);
int sur_lattice_fwd_f32(const float *G, const float *q, const int *ant, int B, int K, int NR, int D, int T, int S,
                        int J, int moff, float *y, void *stream);
/* hi[i] = bf16(x[i]), lo[i] = bf16(x[i] - hi[i]), i < n: x = hi + lo to about
   2^-17 relative, so products of split operands on the bf16 tensor cores
   (hi hi + hi lo + lo hi, f32 accumulation) carry nearly f32 precision. */
int sur_split_bf16(const float *x, void *hi, void *lo, long long n, void *stream);
int sur_lattice_bwd(const float *dy, const float *q, const int *ant, int B, int K, int NR, int D, int T, int S,
                    int J, int moff, float *dG, void *stream);
int sur_lattice_weights(const void *G, const int *ant, int A, int K, int NR, int D, int T, int S, int J, int moff,
                        void *W, void *stream);
/* The same weights K-major, as the B operand of the tcgen05 GEMM:
   W[a][t][koff + k] (bf16, row stride ldw >= koff + K; other columns left as
   they are).  FDTD_ERR_ARG for bad sizes. */
int sur_lattice_weights_kmajor(const void *G, const int *ant, int A, int K, int NR, int D, int T, int S, int J,
                               int moff, void *W, int ldw, int koff, void *stream);
/* out[r][0..K) = out[r][K..2K) = hi(x[r]), out[r][2K..3K) = lo(x[r]) (the
   split of sur_split_bf16), out[r][3K..ld) = 0; x f32 [rows][K], out bf16
   [rows][ld], ld >= 3K: the A operand of [hi, hi, lo] [W_hi; W_lo; W_hi]. */
int sur_split3_bf16(const float *x, int rows, int K, void *out, int ld, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SURROGATE_GB300_H */
