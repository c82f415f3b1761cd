// The FFT lengths compiled into this build, as X-macro entries (N, N1, N2).
#pragma once
#define MOCO_FOR_EACH_FFT_SIZE(X) \
    X(48) X(64) X(96) X(128) X(144) X(160) X(192) X(256) X(288) X(320) X(384) X(512) X(576)
