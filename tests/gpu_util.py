"""Helpers shared by the GPU parity tests (no reconstruction arithmetic here)."""
import numpy as np


def rel_l2(got, ref):
    """||got - ref|| / ||ref||; complex inputs compare as complex."""
    cpx = np.iscomplexobj(got) or np.iscomplexobj(ref)
    got = np.asarray(got, dtype=np.complex128 if cpx else np.float64)
    ref = np.asarray(ref, dtype=np.complex128 if cpx else np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / den) if den > 0 else float(np.linalg.norm(got))


def same_peak(got, ref, rtol=1e-6):
    """Identical global argmax; a different index is accepted only when the
    oracle's value there ties its maximum to within rtol (several voxels are
    then equally correct)."""
    ig = int(np.argmax(got))
    ir = int(np.argmax(ref))
    if ig == ir:
        return True
    r = np.asarray(ref).reshape(-1)
    return abs(r[ig] - r[ir]) <= rtol * abs(r[ir])


def local_peaks_agree(got, ref, centers, half=3):
    """Inside a +-half window around each centre, the argmax is the same voxel."""
    for c in centers:
        sl = tuple(slice(max(0, int(v) - half), int(v) + half + 1) for v in c)
        g, r = got[sl], ref[sl]
        if g.size == 0:
            continue
        if np.unravel_index(np.argmax(g), g.shape) != np.unravel_index(np.argmax(r), r.shape):
            return False
    return True


def to_device(H, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(H), dtype=torch.float64).to(dtype).cuda().contiguous()


def exact_input(H, dtype):
    """The values the device sees after conversion to the storage type, in float64."""
    import torch
    return torch.as_tensor(np.ascontiguousarray(H), dtype=torch.float64).to(dtype).to(torch.float64).numpy()
