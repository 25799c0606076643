"""GB300-native exact Gaussian elimination with transformation over GF(p)
(arXiv 1806.04211).  The compute runs in libgfe.so (CUDA, sm_103a); see
`gfe` for the binding and `synth` for the seeded inputs."""
