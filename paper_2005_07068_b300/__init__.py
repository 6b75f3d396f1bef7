"""B300-native hypothesis scoring for the model-based 26-DOF hand tracker
(arxiv 2005.07068): FK, FP32 analytic ray-cast depth render, the Eq. 4-5 cost
and the PSO step, as hand-written sm_103a CUDA kernels behind a C-ABI."""
