/*
 * spectra.h -- spectra of detector traces (libfdtd_gb300.so).
 *
 * Sec. V reads the detector fields as spectra E_omega: at the Cherenkov angle
 * for several distances R, as angular distributions, and against the
 * far-field formula eq. 1d_appro.  The Fourier convention is that of
 * eq. GreenMethod, whose time factor is exp(+i omega t'):
 *
 *     E_omega(f) = dt * sum_{m=0}^{count-1} g_m x_{first+m} exp(i 2 pi f t_{first+m}),
 *     t_n = t0 + n dt,        x_n = sum_c a_c X[n][c],
 *
 * over a gate of `count` samples from sample `first` of each trace, g the
 * Tukey window of taper fraction alpha (u = m / (count - 1); g = (1 -
 * cos(2 pi u / alpha)) / 2 for u < alpha / 2, g = 1 up to u = 1 - alpha / 2,
 * mirrored above; alpha = 0 is the rectangular gate, count = 1 gives g = 1).
 * The detectors record (E_z, E_r); the field along theta-hat of a spherical
 * frame whose polar axis is the shower axis is a = (-sin theta, cos theta).
 *
 * The phase 2 pi f t_n is carried in 64-bit fixed point (the fraction of a
 * cycle), so it stays exact over any trace length; the sums run in float32
 * within a thread and in float64 across threads.  Status codes as in fdtd.h.
 */
#ifndef SPECTRA_GB300_H
#define SPECTRA_GB300_H

#include "fdtd.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * traces: device pointer, float32 [n_traces][n_t][n_comp] -- the layout that
 *   fdtd_probes and cyl_probes write (n_comp = 2, n_t = max_steps, sample s
 *   taken at time (s + 1) dt);
 * coef: host, double [n_traces][n_comp], or NULL for a = (1, 0, ...);
 * gate: host, int [n_traces][2] (first, count), 0 <= first, 0 <= count,
 *   first + count <= n_t, or NULL for (0, n_t) on every trace;
 * taper: alpha in [0, 1];  dt > 0 and t0: the sample times;
 * freq: host, double [n_freq], Hz (any sign);
 * out: float32 [n_traces][n_freq][2] (re, im): a device pointer
 *   (on_device = 1; the call is asynchronous on `stream`) or a host pointer
 *   (on_device = 0; the call synchronises);
 * stream: a cudaStream_t, or NULL for the legacy default stream.
 * Nothing is kept between calls; the caller owns every buffer.
 * FDTD_ERR_ARG for a null pointer, n_traces, n_t or n_freq < 1, n_comp
 * outside 1..4, a gate outside its trace, taper outside [0, 1], dt <= 0 or a
 * number that is not finite; FDTD_ERR_OOM; FDTD_ERR_CUDA.
 */
int fdtd_trace_spectrum(const float *traces, int n_traces, int n_t, int n_comp,
                        const double *coef, const int *gate, double taper,
                        double dt, double t0, const double *freq, int n_freq,
                        float *out, int on_device, void *stream);

/*
 * Weights of the theta-hat component for fdtd_trace_spectrum (Sec. V reads
 * the radiation field, which lies along theta-hat of a spherical frame whose
 * polar axis is the shower axis): E_theta = E_r cos(theta) - E_z sin(theta),
 * so coef[2t] = -sin(theta[t]) (E_z, trace component 0) and coef[2t+1] =
 * cos(theta[t]) (E_r, component 1).  theta: host, n radians; coef: host,
 * n x 2 doubles.  FDTD_ERR_ARG for a null pointer, n < 1 or a theta that is
 * not finite.
 */
int fdtd_theta_coef(const double *theta, int n, double *coef);

#ifdef __cplusplus
}
#endif

#endif /* SPECTRA_GB300_H */
