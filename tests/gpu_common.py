"""Shared helpers for the GPU parity tests (CUDA path vs FP64 oracle)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def device_tracks(tr, torch, device="cuda"):
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device)
    return dict(n_tracks=tr.n_tracks, n_steps=tr.n_steps, n_out=tr.n_out, dt=tr.dt, charge=1.0,
                x=dev(tr.x), y=dev(tr.y), z=dev(tr.z), vx=dev(tr.vx), vy=dev(tr.vy), vz=dev(tr.vz),
                q=dev(tr.charge))
