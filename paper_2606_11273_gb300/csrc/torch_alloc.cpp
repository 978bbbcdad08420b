// Adapter from lmfs_params.dev_alloc / dev_free to PyTorch's CUDA caching
// allocator, so that a handle created from Python can take all of its device
// memory from the same cache as the caller's tensors.  Plain C entry points:
// the library calls them from any of its threads without the Python
// interpreter (no GIL).  Allocation happens on the current device, which the
// library sets to the handle's device before every call that allocates; the
// block is associated with the handle's stream, where the library uses it.
#include <c10/cuda/CUDACachingAllocator.h>
#include <cuda_runtime.h>

extern "C" void* lmfs_torch_alloc(size_t bytes, void* stream, void*) {
  try {
    return c10::cuda::CUDACachingAllocator::raw_alloc_with_stream(bytes, static_cast<cudaStream_t>(stream));
  } catch (...) {
    return nullptr;   // the library reports LMFS_ERR_NOMEM
  }
}

extern "C" void lmfs_torch_free(void* ptr, void*, void*) {
  try {
    c10::cuda::CUDACachingAllocator::raw_delete(ptr);
  } catch (...) {
  }
}
