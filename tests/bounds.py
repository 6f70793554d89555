"""The stated relative error bounds of the reduced-precision forms, per order p: Eq. 16 on the
check potential (and on the locals through the check potential they reproduce) against the FP64
definition. The GPU parity tests hold every form to these; the library states the same table
(m2l_stated_bound, checked equal in tests/test_capi_host.py).

Largest values measured per p = 4, 6, 8, 10 on depth-3 trees over densities uniform in [0,1),
uniform in [-1,1], Gaussian, and physical multipoles (P2M + M2M of a seeded cloud), with at
least a factor 1.8 of margin:
  FFT FP32     3.9e-7, 3.9e-7, 5.1e-7, 5.3e-7    -> 1e-6
  FFT TF32x3   the same on levels below 5; tensor-core levels (level 5, signed densities,
               p = 4, 6, 8): 1.6e-7, 2.2e-7, 2.6e-7                  -> 1e-6
  BLAS TF32x3  5.2e-7, 1.4e-6, 1.1e-6, 1.3e-6    -> 1e-6 at p <= 4, else 3e-6
  BLAS FP32    1.5e-6, 3.1e-6, 2.4e-6, 1.9e-6    -> 3e-6 at p <= 4, else 6e-6
  BLAS BF16x3  5.5e-6, 5.3e-6, 5.0e-6, 5.9e-6    -> 1.2e-5
"""


def stated(form: str, precision: str, p: int) -> float:
    if precision == "fp64":
        return 1e-11 if p >= 8 else 1e-12
    if form == "fft":
        return 1e-6
    if precision == "tf32x3":
        return 1e-6 if p <= 4 else 3e-6
    if precision == "fp32":
        return 3e-6 if p <= 4 else 6e-6
    return 1.2e-5
