"""libtor: exact Torontonians on GB300 (sm_103a) by the recursive subset-tree method
of arXiv 2109.04528.  The compute path lives in the CUDA library built from
``csrc/``; this package is its thin ctypes binding."""
from .binding import (TorError, Context, TorResult, tor_create, tor_destroy, tor_eval, tor_eval_batch,
                      tor_submit, tor_poll, tor_strerror, load_library, library_path)

__all__ = ["TorError", "Context", "TorResult", "tor_create", "tor_destroy", "tor_eval",
           "tor_eval_batch", "tor_submit", "tor_poll", "tor_strerror", "load_library", "library_path"]
