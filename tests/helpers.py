"""Shared helpers of the GPU tests: uploads in the canonical layouts, precision casts of
vectors as the library stores them, and error norms."""
import numpy as np

PREC_NAMES = ("f64", "f32", "bf16", "f16")


def rel_l2(got, ref):
    got = np.asarray(got)
    ref = np.asarray(ref)
    return float(np.linalg.norm((got - ref).reshape(-1)) / np.linalg.norm(ref.reshape(-1)))


def to_device_vec(v, prec):
    """complex128 numpy (..., 3) -> CUDA tensor in the library's canonical vector format."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(v))
    if prec == "f64":
        return t.cuda()
    if prec == "f32":
        return t.to(torch.complex64).cuda()
    real = torch.view_as_real(t)
    dt = torch.bfloat16 if prec == "bf16" else torch.float16
    return real.to(dt).contiguous().cuda()


def from_device_vec(t):
    """Inverse of to_device_vec: CUDA tensor -> complex128 numpy."""
    import torch
    t = t.detach().cpu()
    if t.is_complex():
        return t.to(torch.complex128).numpy()
    r = t.to(torch.float64).numpy()
    return r[..., 0] + 1j * r[..., 1]


def empty_vec(shape, prec):
    import torch
    if prec == "f64":
        return torch.empty(shape, dtype=torch.complex128, device="cuda")
    if prec == "f32":
        return torch.empty(shape, dtype=torch.complex64, device="cuda")
    dt = torch.bfloat16 if prec == "bf16" else torch.float16
    return torch.empty(tuple(shape) + (2,), dtype=dt, device="cuda")


def store_tolerance(vec_prec):
    """Relative L2 bound for a Dslash output stored in ``vec_prec`` against the FP64 oracle
    applied to the same (already rounded) links and input: one round-to-nearest of each
    output real (unit roundoff 2^-p) plus FP32 accumulation of 16 terms."""
    u = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}[vec_prec]
    acc = 1e-13 if vec_prec == "f64" else 1e-5
    return u + acc
