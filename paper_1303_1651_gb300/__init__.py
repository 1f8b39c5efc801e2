"""GB300-native sparse x sparse product C = A*B on CSR matrices (int32 indices, float64 values).

The method is the row-major (Gustavson) spMMM analysed in Scharpff, Iglberger,
Hager and Ruede, "Model-guided Performance Analysis of the Sparse
Matrix-Matrix Multiplication" (arXiv:1303.1651), re-designed as sm_103a CUDA
kernels behind the C ABI in include/spgemm_gb300.h.

Submodules:
  binding  -- ctypes binding of the C ABI (loads the CUDA library; no CPU fallback), and
              spgemm(A, B), the product of torch sparse CSR/CSC tensors
  synth    -- seeded synthetic inputs (FD 5-point Laplacian, random k per row, batches)
  roofline -- bytes/flops accounting of the product and the paper's balance model
  build    -- nvcc build of the library
  autograd -- torch.autograd function over the product (values of A and B)
  batched  -- many independent products as one block-diagonal product, replayed as a CUDA graph
  tune     -- per-workload choice of row-class options
  ranks    -- host-side helpers for one process per GPU (max over ranks, contiguous shards)
"""
__version__ = "1.0.0"


def __getattr__(name):
    import importlib
    if name == "spgemm":
        return importlib.import_module(".binding", __name__).spgemm
    if name in ("binding", "synth", "build", "roofline", "autograd", "batched", "tune", "ranks"):
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
