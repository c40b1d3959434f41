"""Helpers for the GPU tests: seeded inputs, upload/download, error metrics."""
import numpy as np

from tests._qlayout import planes_to_comp


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def to_host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel_fro(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm((x - ref).ravel()) / max(np.linalg.norm(ref.ravel()), 1e-300))


def assert_close(gpu_planes, ref_comp, rel_tol, elem_tol, what=""):
    """Element-by-element check of a GPU result (plane layout) against an FP64
    oracle result (component layout): relative Frobenius error <= rel_tol and
    every |x - ref| <= elem_tol * rms(ref)."""
    got = planes_to_comp(gpu_planes)
    ref = np.asarray(ref_comp, dtype=np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    assert np.all(np.isfinite(got)), f"{what}: non-finite output"
    rf = rel_fro(got, ref)
    rms = float(np.sqrt(np.mean(ref * ref))) if ref.size else 0.0
    worst = float(np.max(np.abs(got - ref))) if ref.size else 0.0
    assert rf <= rel_tol, f"{what}: relative Frobenius error {rf:.3e} > {rel_tol:.1e}"
    assert worst <= elem_tol * max(rms, 1e-30), f"{what}: max abs error {worst:.3e} > {elem_tol:.1e} * rms {rms:.3e}"
    return rf
