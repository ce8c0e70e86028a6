"""The air-filled guide of the paper's Sec. 5.2.1 on the GPU path.  The paper
Fourier-transforms E on the guide's central line and compares the
attenuation alpha(f) with imag sqrt(w^2 mu0 eps0 - (pi/W)^2) and the cutoff
with c/(2W) = 10.03 GHz.  Here each frequency gets its own narrow-band drive
(a 0.8 ns Gaussian envelope, so nothing reaches the cutoff region, whose
group velocity vanishes); three E_y probes on the central line are
demodulated at the drive frequency over whole periods around the envelope's
peak, and the probe-to-probe ratio gives beta above cutoff and alpha below."""
import numpy as np
import pytest

import paper_2103_12819_b300 as mmx
import workloads as W

pytestmark = pytest.mark.gpu

C0 = 299792458.0
WIDTH = 14.95e-3
FC = C0 / (2 * WIDTH)
TP = 0.8e-9


def _amplitudes(f0, z_probes):
    """Complex amplitude at f0 of E_y on the axis at each probe plane, each
    demodulated over whole periods centred on the envelope's peak at that
    plane (source peak 3 Tp plus the TE10 group delay; no delay below
    cutoff, where the field is evanescent)."""
    w = W.air_guide(f0=f0, tp=TP)
    vg = C0 * np.sqrt(max(0.0, 1.0 - (FC / f0) ** 2))
    z_src = w.sources[0].k
    t_pk = [3 * TP + ((z - z_src) * w.d[2] / vg if vg > 0 else 0.0) for z in z_probes]
    nper = int(np.floor(0.3e-9 * f0))          # whole periods in ~0.3 ns
    m = int(round(nper / (f0 * w.dt)))
    steps = int(np.ceil(max(t_pk) / w.dt)) + m
    s = mmx.from_workload(w, prec=mmx.FP32, path=mmx.PATH_FUSED)
    for z in z_probes:
        s.add_probe(1, 37, 25, z)            # E_y edge nearest the guide axis
    s.step(steps)
    assert s.sync(check=False) == 0, s.last_error()
    sig = s.get_probes()
    s.close()
    t = (np.arange(steps) + 1) * w.dt          # row r holds E^(r+1)
    amp = np.zeros(len(z_probes), dtype=complex)
    for p, tp_ in enumerate(t_pk):
        r0 = int(round(tp_ / w.dt)) - m // 2
        sl = slice(r0, r0 + m)
        amp[p] = np.sum(np.exp(-2j * np.pi * f0 * t[sl]) * sig[sl, p])
    return amp, w.d[2]


@pytest.mark.parametrize("f0", [11.0e9, 12.0e9, 13.0e9])
def test_propagation_constant_and_cutoff(f0):
    """Above cutoff: beta from the phase between probes 100 cells apart
    matches sqrt((w/c)^2 - (pi/W)^2) to 1%, and f_c = sqrt(f^2 - (beta c/2pi)^2)
    is c/(2W) to 0.5%; the amplitude is unattenuated to 2%."""
    zp = (150, 250, 350)
    amp, dz = _amplitudes(f0, zp)
    beta_th = np.sqrt((2 * np.pi * f0 / C0) ** 2 - (np.pi / WIDTH) ** 2)
    for a, b in ((0, 1), (1, 2)):
        r = amp[b] / amp[a]
        L = (zp[b] - zp[a]) * dz
        # the phase advances by beta L, possibly more than 2 pi: take the
        # branch nearest the theory (which only picks the multiple of 2 pi)
        ph = -np.angle(r)
        k = np.round((beta_th * L - ph) / (2 * np.pi))
        beta = (ph + 2 * np.pi * k) / L
        fc = np.sqrt(f0 ** 2 - (beta * C0 / (2 * np.pi)) ** 2)
        print("f0 %.1f GHz probes %d-%d: beta/beta_th %.5f  f_c %.4f GHz  |r| %.4f"
              % (f0 / 1e9, a, b, beta / beta_th, fc / 1e9, abs(r)))
        assert abs(beta / beta_th - 1) < 0.01
        assert abs(fc / FC - 1) < 5e-3
        assert abs(abs(r) - 1) < 0.02


@pytest.mark.parametrize("f0", [8.5e9, 9.3e9])
def test_attenuation_below_cutoff(f0):
    """Below cutoff the drive decays away from the source: alpha from the
    amplitude ratio of probes 40 cells apart matches the paper's
    imag sqrt(w^2 mu0 eps0 - (pi/W)^2) to 5%."""
    zp = (40, 80)
    amp, dz = _amplitudes(f0, zp)
    alpha = -np.log(abs(amp[1] / amp[0])) / ((zp[1] - zp[0]) * dz)
    alpha_th = np.sqrt((np.pi / WIDTH) ** 2 - (2 * np.pi * f0 / C0) ** 2)
    print("f0 %.1f GHz: alpha %.2f /m, theory %.2f /m" % (f0 / 1e9, alpha, alpha_th))
    assert abs(alpha / alpha_th - 1) < 0.05
