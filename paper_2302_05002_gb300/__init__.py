"""GB300-native construction of the FastPoints (arxiv 2302.05002) octree hot
path: bounds, hash preview, count grid, chunk merge, stable distribution,
per-chunk octrees stitched into a shallow LOD octree.  All stages are CUDA
kernels for sm_103a behind the C ABI in include/fastpoints.h; this package is
its Python binding (``fastpoints``) and in-tree build (``build``)."""
__all__ = ["fastpoints", "build"]
