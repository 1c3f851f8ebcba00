"""Helpers for the GPU tests: column-major device buffers and tolerances."""
import numpy as np

EPS64 = float(np.finfo(np.float64).eps)
EPS32 = float(np.finfo(np.float32).eps)


def dev_colmajor(torch, M, ld=None, dtype=None, fill=0.0):
    """Device buffer holding M column-major with leading dimension ld.
    Returns the backing tensor (shape (cols, ld), row-major = column-major)."""
    M = np.asarray(M)
    rows, cols = M.shape
    ld = ld or max(rows, 1)
    dt = dtype or (torch.float64 if M.dtype == np.float64 else torch.float32)
    buf = torch.full((max(cols, 1), ld), fill, dtype=dt)
    if rows and cols:
        buf[:cols, :rows] = torch.from_numpy(np.ascontiguousarray(M.T)).to(dt)
    return buf.cuda()


def host_colmajor(buf, rows, cols):
    """Read back rows x cols of a column-major device buffer from dev_colmajor."""
    return np.asfortranarray(buf.cpu().numpy()[:cols, :rows].T.astype(np.float64))


def factor_tolerance(n, kappa=10.0, eps=EPS64):
    """Elementwise tolerance (relative to max |L|) between two backward-stable
    Cholesky factors of the same matrix: each is within ~n u kappa of the
    exact factor to first order, so their difference within twice that, with
    a factor 4 of headroom for the constant."""
    return 8.0 * max(n, 1) * eps * kappa
