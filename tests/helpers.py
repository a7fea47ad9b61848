"""Conversions between oracle arrays and the library's column-major buffers."""
import numpy as np

from paper_2608_17123_b300.inputs import to_colmajor, from_colmajor


def img_to_dev(X, dtype):
    import torch
    return torch.from_numpy(to_colmajor(X)).to(device="cuda", dtype=dtype).reshape(-1).contiguous()


def dev_to_img(t, m):
    return from_colmajor(t.detach().double().cpu().numpy().reshape(-1), m)


def planes_to_dev(qx, qy, dtype):
    """(qx: (m-1) x m, qy: m x (m-1)) -> padded planes [x | y], each m x m column-major."""
    import torch
    m = qy.shape[0]
    px = np.zeros((m, m))
    px[: m - 1, :] = qx
    py = np.zeros((m, m))
    py[:, : m - 1] = qy
    buf = np.concatenate([to_colmajor(px).ravel(), to_colmajor(py).ravel()])
    return torch.from_numpy(buf).to(device="cuda", dtype=dtype).contiguous()


def dev_to_planes(t, m):
    a = t.detach().double().cpu().numpy().reshape(-1)
    px = from_colmajor(a[: m * m], m)
    py = from_colmajor(a[m * m:], m)
    return px[: m - 1, :], py[:, : m - 1], px[m - 1, :], py[:, m - 1]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))
