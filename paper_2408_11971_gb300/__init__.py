"""HoSZp on GB300: homomorphic error-bounded lossy compression (arXiv 2408.11971).

A thin Python binding over ``libhoszp.so`` (the hand-written sm_103a CUDA kernels
behind the C ABI of ``include/hoszp.h``). The functions here only marshal
arguments: device memory comes from torch tensors, streams from torch streams,
and every step of the codec and of the operators runs in the library's kernels.
There is no CPU fallback: importing works without a GPU, but every call needs
the compiled library and a CUDA device, and raises otherwise.

    import torch, paper_2408_11971_gb300 as hz
    c = hz.compress(x_cuda, eb=1e-3, mode="rel")   # uint8 tensor (the stream)
    m = hz.mean(c)                                 # Sec. V-B, from the stream
    z = hz.add(c, hz.negate(c))                    # Sec. V-A / V-C
    y = hz.decompress(z)
"""
from ._binding import (  # noqa: F401
    HoszpError,
    Context,
    Batch,
    Server,
    STATUS,
    lib_path,
    load_library,
    default_context,
    compress_bound,
    compress,
    decompress,
    negate,
    add_scalar,
    sub_scalar,
    mul_scalar,
    mul_scalar_exact,
    add,
    sub,
    hadamard,
    mean,
    var,
    std,
    cov,
    block_means,
    sums,
    finish_sums,
    concat,
    batch_compress,
    header,
    fop_axpb,
    fop_add,
    fop_moments,
)

__all__ = [
    "HoszpError", "Context", "Batch", "Server", "STATUS", "lib_path", "load_library",
    "default_context", "compress_bound", "compress", "decompress", "negate", "add_scalar",
    "sub_scalar", "mul_scalar", "mul_scalar_exact", "add", "sub", "hadamard", "mean", "var",
    "std", "cov", "block_means", "sums", "finish_sums", "concat", "batch_compress", "header", "fop_axpb", "fop_add", "fop_moments",
]
